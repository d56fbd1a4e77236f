// Internal declarations shared by the ffsyrk translation units.
//
// Data layout in HBM (one call of Algorithm 2 with L levels, n×k padded to
// n_pad×k_pad so that every level splits evenly):
//   * node matrices (uint32 residues in [0,p)): depth 0 is the user's A
//     (read with virtual zero padding); X11 and X12 children are strided views
//     of their parent; only S3 children are materialised;
//   * operand arenas, one per leaf K length: arena j (1 ≤ j ≤ L) holds the
//     general-product operands of depth j−1 (X22, S4, S1, S2 per node) and,
//     for j = L, the 3^L syrk-leaf operands.  Each operand is D digit planes
//     of R_pad×K_pad elements, plane after plane (bf16 digits for the tensor
//     leaf; one plane of uint32 residues for the int64 leaf);
//   * product buffers: leaf syrk results and per-depth node results (lower
//     triangle used), P3/P4 per node (full), all uint32 residues.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

namespace fsk {

constexpr int kMaxLevels = 6;
constexpr int kMaxDigits = 3;
constexpr int kMaxPlanes = 6;  // digit planes per operand: D, plus D(D−1)/2 digit sums

// Barrett-style reduction constants for p < 2^24.
struct ModP {
    uint32_t p;
    uint32_t half;     // (p−1)/2: residues above it are negative in signed form
    uint32_t barrett;  // floor(2^32 / p)
    uint32_t dbase;    // digit base of the tensor-core operands (see DigitScheme)
    float dinv;        // 1 / dbase
};

// Multiplication by a constant w < p with Shoup's precomputed quotient
// w_sh = floor(w·2^32 / p).
struct MulConst {
    uint32_t w;
    uint32_t w_sh;
};

// How the kernel that writes the caller's C stores a result R (residues in
// [0, p)): mode 0 stores R; mode 1 stores α·R + β·C_old mod p, the update
// C ← α·A·Aᵀ + β·C of Table 4 applied where C is written (same result as
// scaling the products and adding β·C blockwise as that schedule does).
struct OutScale {
    uint32_t mode;
    MulConst alpha, beta;
};
#ifdef __CUDACC__
// x·c mod p for x < 2^32 (Shoup's precomputed quotient c.w_sh = ⌊c.w·2^32/p⌋)
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, MulConst c, uint32_t p) {
    const uint32_t q = __umulhi(x, c.w_sh);
    const uint32_t r = x * c.w - q * p;
    return r >= p ? r - p : r;
}
// α·r + β·old mod p for r, old < p
__device__ __forceinline__ uint32_t scale_out(uint32_t r, uint32_t old, const OutScale &s, uint32_t p) {
    const uint32_t v = mul_shoup(r, s.alpha, p) + mul_shoup(old, s.beta, p);
    return v >= p ? v - p : v;
}
#endif

// The skew-orthogonal Y (Section 3.1): form 0 is i·I; form 1 is the
// interleaved I ⊗ [[a, b], [−b, a]].
struct YConst {
    int form;
    MulConst a;  // i, or a
    MulConst b;  // b (form 1)
};

// Signed digits of the symmetric residue and the per-pair
// chunk lengths that keep every FP32 partial sum an exact integer.
// Residues in signed form s ∈ [−(p−1)/2, (p−1)/2] are written as
// s = Σ_t d_t·base^t with D signed digits, every |d_t| ≤ 256 (exact in bf16).
// The base is 256 (byte digits) unless D = 2 and the top byte digit would
// exceed 128 (primes between 2^16 and 2^17): there a balanced base b ≈ √p
// bounds both digits by b/2 ≤ 256, so that the worst digit pair, and with it
// the shortest exact K-chunk, is no worse than the others (p = 131071:
// base 362, digits ≤ 181, every pair 8 k-blocks per chunk instead of 4 for
// the top pair of byte digits).
//
// Digit products.  Schoolbook: the D² pairs (i, j) of single digit planes,
// X·Zᵀ = Σ b^(i+j)·X_i·Z_jᵀ.  Karatsuba (when every |digit| ≤ 128, so that
// a sum of two digits stays an exact bf16 integer ≤ 256): each operand also
// carries the D(D−1)/2 planes X_i + X_j (i < j), and the D(D+1)/2 products
// P_t = plane_t(X)·plane_t(Z)ᵀ give X·Zᵀ = Σ_t w_t·P_t with
//   w_t = b^(2i) − Σ_{j≠i} b^(i+j) for the single plane t = i,
//   w_t = b^(i+j) for the sum plane of (i, j),
// since X_i·Z_jᵀ + X_j·Z_iᵀ = (X_i + X_j)·(Z_i + Z_j)ᵀ − X_i·Z_iᵀ − X_j·Z_jᵀ.
// Planes: 0..D−1 the digits, then the sums (0,1), (0,2), (1,2).
struct DigitScheme {
    int D;
    int base;                                  // 256, or the balanced base for D = 2
    int ks;                                    // 1: Karatsuba digit products
    int nplanes;                               // planes per operand: D, or D(D+1)/2 with ks
    int max_digit[kMaxPlanes];                 // bound of |plane t| entries
    int chunk_kb[kMaxPlanes][kMaxPlanes];      // K-chunk per plane pair, in k-blocks
    MulConst weight[kMaxPlanes][kMaxPlanes];   // weight of the product of planes (i, j) mod p
    uint32_t offset;                           // a multiple of p ≥ the accumulator bound
    int lazy_units;  // units the epilogue may add (each < 2p) before its uint32 sums need a reduction
};

// ModP of p with the digit base of ds.
inline ModP make_modp(uint32_t p, const DigitScheme &ds) {
    ModP m;
    m.p = p;
    m.half = (p - 1) / 2;
    m.barrett = (uint32_t)((uint64_t(1) << 32) / p);
    m.dbase = (uint32_t)ds.base;
    m.dinv = 1.0f / (float)ds.base;
    return m;
}

// A uint32 matrix view with virtual zero padding beyond (vr, vc).
struct MatView {
    const uint32_t *ptr;
    int64_t ld;
    int64_t vr, vc;
};

// Element types of operand arenas: bf16 signed digits (tensor-core leaf),
// uint32 residues (int64 leaf, and operands split further by Algorithm 1),
// bytes of the two's-complement residue (INT8 leaf: unsigned low digits,
// signed top digit).
enum ArenaKind { ARENA_BF16 = 0, ARENA_U32 = 1, ARENA_I8 = 2, ARENA_BF16_KS = 3 };
// ARENA_BF16_KS: bf16 digit planes followed by the Karatsuba sum planes
// (DigitScheme::ks); the same element type as ARENA_BF16.

struct Arena {
    void *base = nullptr;   // [rows][kpad] elements
    int64_t rows = 0;       // total rows (all operands, all digit planes)
    int64_t kpad = 0;       // padded leaf K (multiple of 64)
    int64_t rpad = 0;       // rows per digit plane of one operand
    int planes = 1;         // digit planes per operand
    int kind = ARENA_BF16;
    int64_t bytes() const {
        return rows * kpad * ((kind == ARENA_BF16 || kind == ARENA_BF16_KS) ? 2 : kind == ARENA_I8 ? 1 : 4);
    }
};

// Destination of one derived operand written by a pre-addition kernel.
struct OperandDst {
    void *arena;       // nullptr = not written
    int64_t row0;      // first row of digit plane 0
    int64_t kpad;      // row length in elements
    int64_t rpad;      // rows per digit plane
    // bf16 digit planes: the arena's norm table ([plane][256-column block],
    // nb blocks per plane; see NormTables), max-accumulated by the writer;
    // nullptr: none
    uint32_t *norm = nullptr;
    int32_t nb = 0;
};

// One node of a recursion depth for the pre-addition kernel.
struct PrepNode {
    MatView X;                  // the node's (padded h×w) matrix
    OperandDst gemm[4];         // X22, S4 (P3 = X22·S4ᵀ) and S1, S2 (P4 = S1·S2ᵀ)
    OperandDst leaf[3];         // X11, X12, S3 as leaf operands (last level)
    uint32_t *s3;               // S3 as uint32 for the next depth (else nullptr)
    int64_t s3_ld;
};

// One matrix to digit-split (classical path; one per problem when batched).
struct DigitizeJob {
    MatView X;
    int64_t rows;
    OperandDst dst;
    int64_t block0;  // first block of this job in a flattened launch (prefix sum)
    // 1: split X·Jᵀ instead of X, J = I ⊗ [[0, −1], [1, 0]]: each column
    // pair (x, y) becomes (−y, x) (the conjugation step of the Hermitian
    // product over F_p[i], Section 3.2)
    int conj;
};

// One post-addition node: combines the five products into the node result.
struct PostNode {
    const uint32_t *P1, *P2, *P5;  // lower h×h (ld = ldr)
    const uint32_t *P3, *P4;       // full h×h (ld = ldg)
    int64_t ldr, ldg;
    uint32_t *out;                 // 2h×2h result
    int64_t ldo;
    int64_t vn;                    // rows/cols of `out` that exist (root: n)
    int upper;                     // write the upper triangle (transposed)
    OutScale scale;                // root node only: how C is updated
};

// One leaf product out = X·Zᵀ mod p (rows × cols) on arena operands.
struct LeafProd {
    int32_t arena;
    int32_t tri;          // entries written: 0 all; 1 lower (c ≤ r); 2 upper (c ≥ r)
    int64_t a_row0, b_row0;
    int64_t rows, cols;   // valid output extent
    int32_t kblocks;      // K_pad / 64
    int32_t nseg;         // segments of the K schedule (see LeafSeg)
    int64_t plane_rows;   // arena rows between consecutive digit planes of an operand
    uint32_t *out;
    int64_t ldo;
    int64_t seg0;         // first segment in the launch's segment table
    OutScale scale;       // a product that writes the caller's C: how it is updated
};

// One step of a tile's K schedule: digit pair (i, j) over k-blocks
// [kb0, kb0 + nkb).  `first` opens a unit: a run of segments of one weight
// class 256^(i+j) accumulated in one FP32 tensor-memory buffer and drained
// once by the epilogue.  Built on the host (build_segments) so the kernels
// carry only an index.
struct LeafSeg {
    int32_t kb0;
    uint16_t nkb;
    uint8_t ij;     // i << 4 | j
    uint8_t first;
};
// The schedule for one product with `kblocks` k-blocks: balanced spans of
// at most min(span_cap, shortest chunk) k-blocks; inside a span the weight
// classes e = i + j in order, the pairs of a class in order; a unit grows
// while its worst-case |sum| Σ kbw·nkb·max|d_i|·max|d_j| stays ≤ bound and
// never crosses a class.  The tensor-core leaf: k-blocks of kbw = 64, bound
// 2^24 (exact FP32), spans ≤ 16; the INT8 leaf: kbw = 128, bound 2^30
// (int32 with room for the reduction's offset), spans ≤ 128.  With units
// from the operands' digits (below) the tensor-core spans are 32 k-blocks
// whatever the shortest worst-case chunk (clip_span false): the worst-case
// units inside a span are as many as before, and the data-driven merge can
// join them across twice the K.
struct SegRule {
    int64_t bound = int64_t(1) << 24;
    int kbw = 64;
    int span_cap = 16;
    bool clip_span = true;  // spans no longer than the shortest worst-case chunk
};
constexpr SegRule kSegTc{};
constexpr SegRule kSegTcData{int64_t(1) << 24, 64, 32, false};
constexpr SegRule kSegI8{int64_t(1) << 30, 128, 128};
void build_segments(const DigitScheme &ds, int kblocks, std::vector<LeafSeg> &out,
                    const SegRule &rule = kSegTc);
// The same into a caller's buffer of `cap` entries: the count, or −1 if it does not fit.
int build_segments_into(const DigitScheme &ds, int kblocks, LeafSeg *out, int cap,
                        const SegRule &rule = kSegTc);

// ---- unit lengths from the operands' digits ----
// The worst-case schedule above bounds a unit's partial sums by
// Σ nkb·kbw·max|d_i|·max|d_j|.  The digits a call actually holds give a
// bound that is never larger: for one pair over a K range, every partial sum
// of Σ_k x_k·z_k, in any order, is at most Σ_k |x_k|·|z_k| ≤
// sqrt(Σ_k x_k²)·sqrt(Σ_k z_k²) (Cauchy–Schwarz), and Σ_k x_k² over a range
// is at most the sum, over the 256-column blocks the range touches, of the
// largest row sum of squares of that plane in the block.  The kernels that
// write the digit planes also take those block maxima per arena and plane
// (OperandDst::norm); before the leaf one pass
// merges consecutive segments of one weight class into one unit while the
// data bound of the unit stays ≤ 2^24 (exact FP32), so uniform residues
// take about one drain per product and 16 k-blocks instead of one per
// 4 k-blocks for the digit-sum products.  The units never outnumber the
// worst-case schedule's (greedy packing of a sequence whose worst-case
// packing is feasible), so the leaf's lazy-sum bound still holds.
constexpr int kNormCols = 256;  // columns per block of the norm tables (4 k-blocks)
struct NormTables {
    uint32_t *base;                   // [arena][plane][block] maxima, zeroed before each call
    int32_t off[kMaxLevels + 1];      // first entry of arena j
    int32_t nb[kMaxLevels + 1];       // blocks per plane of arena j (ceil(kpad / 256))
};
// One K schedule shared by the products whose arenas are in `arenas` (bit j).
struct UnitJob {
    int64_t seg0;
    int32_t nseg;
    uint32_t arenas;
};
// links[s] (one byte per segment of the launch's table): 1 if segment s may
// continue the unit of segment s − 1 (same schedule, same weight class, and
// not the first segment of a shared tile's piece), else 0.

struct LeafTile {
    int32_t prod;
    int32_t tm, tn;
    int32_t cost;
};

// Part of a tile's K schedule, for tiles shared by several CTAs (the tail of
// a launch is split so that every CTA ends at about the same time).  A piece
// covers segments [sx0, sx1) of its product, starting and ending on unit
// boundaries.  A tile split in npieces pieces owns partial-result slots
// slot0 .. slot0 + npieces − 1 and one counter per epilogue warp at
// 8·slot0 + warp; piece j writes its residues to slot slot0 + j, and for each
// warp's rows the piece that finishes them last adds the others' and stores
// them.  slot0 < 0: the piece is the whole tile (stored directly).
struct LeafPiece {
    int32_t sx0, sx1;
    int32_t slot0;
    int16_t j, npieces;
};

// Per-device launch state of a kernel family (dynamic shared-memory opt-in,
// occupancy): cudaFuncSetAttribute applies to the current device only, so a
// launcher keeps one entry per device, filled on its first launch there
// under the slot's mutex (calls may come from several host threads).
constexpr int kMaxDevices = 64;
struct DeviceOnce {
    std::mutex mu;
    bool done[kMaxDevices] = {};
    int value[kMaxDevices] = {};
};
// Run init(&value) once for the current device; returns its error, and the
// stored value through *value.  Devices beyond kMaxDevices are refused.
template <class F>
cudaError_t once_per_device(DeviceOnce &o, int *value, F init) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(o.mu);
    if (!o.done[dev]) {
        int v = 0;
        e = init(&v);
        if (e != cudaSuccess) return e;
        o.value[dev] = v;
        o.done[dev] = true;
    }
    if (value) *value = o.value[dev];
    return cudaSuccess;
}

// ---- launchers (each returns cudaGetLastError() of its launch) ----
// reduce_input: some node views may hold values ≥ p (views of the caller's A)
cudaError_t launch_prep(const PrepNode *nodes_dev, int nnodes, int64_t h, int64_t w,
                        int64_t kpad, ModP mp, YConst y, DigitScheme ds, int arena_kind,
                        bool reduce_input, cudaStream_t st);
// max_rows, max_kpad: the largest rows and padded K over the jobs (njobs ≤ 65535)
cudaError_t launch_digitize(const DigitizeJob *jobs_dev, int njobs, int64_t max_rows,
                            int64_t max_kpad, ModP mp, DigitScheme ds, int arena_kind,
                            cudaStream_t st);
// Digit split of many matrices in one flattened launch: exactly the blocks
// the jobs need (jobs[t].block0 = blocks of jobs 0..t−1; total_blocks in all).
// block_job (optional, device): the job of every block, saving each block a
// binary search over the jobs.
cudaError_t launch_digitize_flat(const DigitizeJob *jobs_dev, int njobs, int64_t total_blocks,
                                 ModP mp, DigitScheme ds, int arena_kind, cudaStream_t st,
                                 const int32_t *block_job = nullptr);
// blocks one job needs in launch_digitize_flat
int64_t digitize_flat_blocks(int64_t rows, int64_t kpad);
// upper: a node writes the upper triangle (transposed); otherwise the
// fused one-pass kernel over lower tile pairs runs
cudaError_t launch_post(const PostNode *nodes_dev, int nnodes, int64_t h, ModP mp,
                        cudaStream_t st, bool upper);
cudaError_t launch_zero_tri(uint32_t *C, int64_t n, int64_t ldc, int upper, cudaStream_t st);
// count uniform residues in [0, p) from a counter hash (the autotuner's operands)
cudaError_t launch_fill_residues(uint32_t *A, int64_t count, uint32_t p, uint64_t seed, cudaStream_t st);
// The `first` flags of every job's segments from the tables (see UnitJob).
cudaError_t launch_unit_schedule(const UnitJob *jobs_dev, int njobs, const NormTables &t,
                                 const uint8_t *links, LeafSeg *segs, const DigitScheme &ds,
                                 cudaStream_t st);
// One operand of a general product L·Rᵀ split by one level of Algorithm 1
// (Winograd's variant of Strassen's product): X is 2hh × 2ww uint32
// residues (row stride ldx, a multiple of 4); side 0 writes the left
// operands of p1..p7, side 1 the right ones, into dst[0..6] (each hh rows).
struct SwPreJob {
    const uint32_t *X;
    int64_t ldx;
    int side;
    OperandDst dst[7];
};
// The post-additions of one level of Algorithm 1: the 7 products p1..p7
// (hh × hh, row stride hh) into C = [[c3, c7], [c4, c5]] (2hh × 2hh, row
// stride 2hh).
struct SwPostJob {
    const uint32_t *P[7];
    uint32_t *C;
};
// out_kind: ARENA_U32 writes uint32 rows (another level follows, or the
// int64 leaf), otherwise the digit planes of the tensor-core leaf
cudaError_t launch_sw_pre(const SwPreJob *jobs_dev, int njobs, int64_t hh, int64_t ww,
                          int64_t kpad, ModP mp, DigitScheme ds, int out_kind, cudaStream_t st);
cudaError_t launch_sw_post(const SwPostJob *jobs_dev, int njobs, int64_t hh, ModP mp,
                           cudaStream_t st);

// Constants of F_p for the scaling planner of Section 5 (from the host).
struct ScaleConst {
    uint32_t p;
    uint64_t minv;   // ⌊(2^64 − 1)/p⌋: Barrett reduction of 64-bit values
    uint32_t q, s;   // p − 1 = q·2^s with q odd
    uint32_t zq;     // z^q, z the least non-square (Tonelli–Shanks)
    uint32_t s_inv;  // 1/z
    uint32_t c_sos;  // √(z − 1), a square because z − 1 < z (Algorithm 3)
    uint32_t inv2;   // 1/2
};
// Device scratch of the scaling planner: W (kk columns, each up to four
// (source, weight) pairs) and per-column state of the k columns of A.
struct ScalePlan {
    int4 *src;       // kk: source columns of A (−1 unused)
    uint4 *w;        // 2·kk: per column four (weight, ⌊weight·2^32/p⌋) pairs
    uint32_t *dbar;  // k: the diagonal after the 2×2 blocks are made diagonal
    uint32_t *ta;    // k: column c of T is ta[c]·e_c + tb[c]·e_mate[c]
    uint32_t *tb;
    int32_t *mate;   // k: the other column of c's 2×2 block, or −1
    uint32_t *flag;  // k: 1 where d̄ is a non-square
    int32_t *ns;     // k: the non-square columns in column order
    int64_t *ns_count;
};
// The planner's kernels: W for B with diagonal d_dev and off-diagonal e_dev
// (device copies of k and k − 1 entries).  Sets bit 2 of *err if a check
// fails (a 2×2 block needing a fifth term, a non-square given to the square
// root, or an odd count of non-squares that kk = k does not admit).
cudaError_t launch_scale_plan(const uint32_t *d_dev, const uint32_t *e_dev, bool has_e, int64_t k,
                              int64_t kk, const ScaleConst &f, const ScalePlan &sp,
                              unsigned int *err, cudaStream_t st);
// Ā = A·W, Ā n × kk with row stride ldb (see k_col_mix)
cudaError_t launch_col_mix(const uint32_t *A, int64_t lda, int64_t n, int64_t kk, const int4 *src,
                           const uint4 *w, uint32_t *B, int64_t ldb, ModP mp, cudaStream_t st);
// the selected triangle for k = 0: zero, or β·C (sc.mode 1)
cudaError_t launch_scale_tri(uint32_t *C, int64_t n, int64_t ldc, int upper, const OutScale &sc,
                             uint32_t p, cudaStream_t st);
cudaError_t launch_leaf_i64_arrays(const LeafProd *prods_dev, const LeafTile *tiles_dev,
                                   int ntiles, const uint32_t *const *arenas_dev,
                                   const int64_t *kpad_dev, ModP mp, cudaStream_t st);

// The tensor-core leaf.  tmaps_dev holds one CUtensorMap (128 B) per arena.
struct TcLaunch {
    const LeafProd *prods;
    const LeafTile *tiles;
    const LeafSeg *segs;
    int ntiles;
    const void *tmaps;        // device array of CUtensorMap, 64-B aligned
    ModP mp;
    DigitScheme ds;
    unsigned int *err;        // device-visible error word (bounded waits)
    unsigned int *tile_ctr;   // device work counter (zeroed before launch)
    // optional work split (1-CTA leaf only): pieces[i] describes tiles[i];
    // entries[e] .. entries[e+1] are the items one CTA takes together
    const LeafPiece *pieces;  // nullptr: every item is a whole tile
    const int32_t *entries;   // nullptr: entry e is item e
    int nentries;
    uint32_t *part;           // partial-result slots, BM·BN residues each
    unsigned int *part_ctr;   // 8 per split tile, zero before the first launch
    int max_units;            // most units (accumulator drains) of any tile's K schedule
    bool scaled;              // a product updates the caller's C (OutScale mode 1)
    bool short_tiles;         // 1-CTA leaf: many tiles of few k-blocks (a batch of small
                              // problems)
    int epi_warps;            // 1-CTA leaf: epilogue warps, 8 or 16 (frequent drains)
};
// Units (segments that open an accumulator) of a K schedule.
int count_units(const LeafSeg *segs, int nseg);
cudaError_t launch_leaf_tc(const TcLaunch &L, int num_sms, cudaStream_t st);
int leaf_tc_bm();
int leaf_tc_bn();
// the same leaf on 256×256 tiles computed by a pair of CTAs (cta_group::2)
cudaError_t launch_leaf_tc2(const TcLaunch &L, int num_sms, cudaStream_t st);
int leaf_tc2_bm();
int leaf_tc2_bn();
int leaf_i64_tile();

// The signed digit scheme (base 256, or a balanced base) and chunk lengths
// the planner uses for p.
DigitScheme digit_scheme_for(uint32_t p);
// The INT8 leaf's digits of p: the D bytes of the two's-complement
// symmetric residue (max_digit 255 below the top digit), weights 256^(i+j)
// mod p, offset the least multiple of p ≥ 2^30.
DigitScheme digit_scheme_i8(uint32_t p);

// The INT8 leaf (kern_leaf_i8.cu): 128×128 tiles, 128-byte k-blocks.
struct I8Launch {
    const LeafProd *prods;
    const LeafTile *tiles;
    const LeafSeg *segs;
    int ntiles;
    const void *tmaps;  // device array of CUtensorMap (uint8 arenas), 64-B aligned
    ModP mp;
    DigitScheme ds;     // digit_scheme_i8
    unsigned int *err;
};
cudaError_t launch_leaf_i8(const I8Launch &L, int num_sms, cudaStream_t st);
int leaf_i8_bm();
int leaf_i8_bn();

// Throughput probe of one arithmetic pipe (see kern_probe.cu): kind 0..4.
cudaError_t launch_probe(int kind, int64_t iters, int blocks, unsigned int *sink, cudaStream_t st);
double probe_macs(int kind, int64_t iters, int blocks);

// A kernel whose bounded wait runs out (after limit_ns) and records it in err.
cudaError_t launch_wait_selftest(unsigned int *err, unsigned long long limit_ns, cudaStream_t st);

// Build the TMA descriptor of an arena: bf16 (box 64 × 128 rows) or uint8
// (INT8 leaf, box 128 × 128 rows), 128B swizzle.
bool encode_arena_tmap(const Arena &a, void *tmap_out /* 128 B */);

}  // namespace fsk
