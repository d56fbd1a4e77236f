/*
 * ffsyrk -- C = A·Aᵀ over a prime field F_p on one GB300 GPU (sm_103a).
 *
 * Implements Algorithm 2 ("syrk") of Dumas, Pernet and Sedoglavic, "On Fast
 * Multiplication of a Matrix by its Transpose" (arXiv 2001.04109, Section 3):
 * per recursion level 4 block pre-additions (two of them times a
 * skew-orthogonal Y), 3 recursive products (P1, P2, P5), 2 general products
 * (P3, P4) and the post-additions U1..U5, down to classical leaves.  All
 * arithmetic is exact integer arithmetic mod p; the result is bit-exact.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major.  A is n×k with leading dimension lda ≥ max(1,k);
 *   C is n×n with ldc ≥ max(1,n).  Any lda/ldc is accepted (no alignment
 *   requirement).  Entries of A may be any uint32; they are reduced mod p.
 * - A and C are DEVICE pointers owned by the caller (ffsyrk_host alone takes
 *   host matrices; the diagonals of the scaled products are host arrays).
 *   The library never frees or retains them beyond the call.
 * - uplo = FFSYRK_LOWER writes C[i][j] = (A·Aᵀ)[i][j] mod p for j ≤ i
 *   (canonical, in [0, p)); FFSYRK_UPPER writes the same values at C[j][i].
 *   The other strict triangle of C is never read or written (ffsyrk_host
 *   returns the whole host matrix, zeros there).
 * - n = 0 is a no-op; k = 0 writes zeros to the selected triangle.
 * - p must be an odd prime with 3 ≤ p < 2^24 (FFSYRK_ERR_NOT_PRIME for a
 *   composite, FFSYRK_ERR_UNSUPPORTED_P for 2 or p ≥ 2^24).
 * - Work is enqueued asynchronously on `stream` (NULL = legacy default
 *   stream).  Argument errors are returned synchronously before anything is
 *   enqueued.  A device-side failure (a bounded wait that ran out) is
 *   recorded in the plan and reported by ffsyrk_sync_status() or by the
 *   next call with the same plan as FFSYRK_ERR_TIMEOUT.
 * - The calling thread's current CUDA device is the device used.
 */
#ifndef FFSYRK_H
#define FFSYRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so users need no CUDA header. */
struct CUstream_st;
typedef struct CUstream_st *ffsyrk_stream_t;

typedef enum {
    FFSYRK_SUCCESS = 0,
    FFSYRK_ERR_INVALID_ARG = 1,   /* bad size, stride, pointer or option    */
    FFSYRK_ERR_NOT_PRIME = 2,     /* p is composite                          */
    FFSYRK_ERR_UNSUPPORTED_P = 3, /* p = 2 or p ≥ 2^24                       */
    FFSYRK_ERR_ALLOC = 4,         /* device or host workspace allocation     */
    FFSYRK_ERR_CUDA = 5,          /* a CUDA runtime call failed              */
    FFSYRK_ERR_TIMEOUT = 6,       /* a device-side bounded wait ran out      */
    FFSYRK_ERR_ARCH = 7,          /* the device is not sm_103 (GB300)        */
    FFSYRK_ERR_TOO_LARGE = 8      /* shape exceeds the plan or a hard limit  */
} ffsyrk_status_t;

typedef enum { FFSYRK_LOWER = 0, FFSYRK_UPPER = 1 } ffsyrk_uplo_t;

/* Which kernel computes the leaf products (the 3^L syrk leaves and the
 * general products of every level). */
typedef enum {
    FFSYRK_LEAF_AUTO = 0,    /* the tensor-core leaf                          */
    FFSYRK_LEAF_TC_BF16 = 1, /* tcgen05.mma kind::f16 on exact 8-bit digits,
                                FP32 TMEM accumulators, reduction per K-chunk */
    FFSYRK_LEAF_I64 = 2,     /* CUDA-core 32×32→64-bit multiply-add leaf      */
    FFSYRK_LEAF_I8 = 3       /* warp-level INT8 tensor path (mma.sync
                                m16n8k32, u8/s8 bytes of the two's-complement
                                residue, int32 register accumulators,
                                reduction per weight class; Section 4.2)     */
} ffsyrk_leaf_t;

#define FFSYRK_LEVELS_AUTO (-1)

/* Planning options.  Fill with ffsyrk_options_default() and change what you
 * need; a NULL options pointer means the defaults. */
typedef struct {
    int32_t leaf;   /* ffsyrk_leaf_t (default FFSYRK_LEAF_AUTO)                 */
    int32_t levels; /* FFSYRK_LEVELS_AUTO (default): chosen from the shape;
                       0 = classical SYRK from the same leaves (no Algorithm 2
                       level); L >= 1 = L levels of Algorithm 2, L <= 6        */
    int32_t tile_ctas; /* tensor-core leaf tiles: 0 = choose from the shape;
                          1 = 128×256 tiles on one SM; 2 = 256×256 tiles on a
                          pair of SMs (tcgen05 cta_group::2)                    */
    int32_t autotune;  /* 1 (with levels = FFSYRK_LEVELS_AUTO and tile_ctas = 0):
                          ffsyrk_plan times every candidate depth and tile
                          variant (and, for one-SM tiles, 8 or 16 epilogue
                          warps) at max_n × max_k on synthetic data in its own
                          workspace and keeps the fastest.  Results are cached
                          per process and, if the environment variable
                          FFSYRK_TUNE_CACHE names a file, in that file.
                          0: depth from the built-in cost model.            */
    int32_t winograd;  /* levels of Algorithm 1 (Winograd's variant of
                          Strassen's product, Section 2) for the two general
                          products P3, P4 of depth d, never more than
                          L − 1 − d (the paper's G-i variants, Section 4.2,
                          take exactly that): −1 (default) = as many as the
                          built-in cost model finds worth it; 0 = none;
                          w ≥ 1 = min(w, L − 1 − d) at every depth d.       */
    int32_t digit_products; /* tensor-core leaf: how the digit planes of the two
                          operands are multiplied (all exact).  0 (default):
                          Karatsuba where it applies, else schoolbook;
                          1 = schoolbook, the D² products X_i·Z_jᵀ;
                          2 = Karatsuba: when every digit is at most 128 in
                          magnitude (byte digits, e.g. p = 65521, 8388593),
                          each operand also carries the D(D−1)/2 planes
                          X_i + X_j and D(D+1)/2 products replace the D²
                          (3 for 4, 6 for 9); elsewhere the same as 1.      */
    int32_t epilogue_warps; /* one-SM tensor-core leaf: warps that drain the
                          accumulators, 8 or 16; 0 (default) = 16 with
                          Karatsuba digit products (frequent drains), else 8 */
    int32_t unit_bounds; /* tensor-core leaf: how long an FP32 accumulator runs
                          before the epilogue reduces it (a unit; every unit
                          is exact, its partial sums ≤ 2^24 in magnitude).
                          0 (default): from the digits of the call's
                          operands -- before the leaf, a pass takes per digit
                          plane and 256-column block the largest row sum of
                          squares, and consecutive segments of one weight
                          class share a unit while Cauchy–Schwarz on those
                          sums keeps the unit ≤ 2^24 (never more units than
                          1); 1: from the largest digit magnitudes alone
                          (K-chunk × max|d_i| × max|d_j| ≤ 2^24).          */
    int32_t reserved;    /* must be zero                                       */
} ffsyrk_options_t;

/* The defaults: automatic leaf, recursion depth and Winograd levels. */
void ffsyrk_options_default(ffsyrk_options_t *opts);

/* Opaque plan: the field constants (p, Y), the digit scheme, the recursion
 * depth and the device workspace for problems up to max_n × max_k.  Owned by
 * the caller; release with ffsyrk_plan_destroy().  A plan belongs to the
 * device that was current when it was made; it is not thread-safe (use one
 * plan per host thread, or serialise calls). */
typedef struct ffsyrk_plan_st *ffsyrk_plan_t;

/* Make a plan for p and problems with n ≤ max_n, k ≤ max_k.  Validates p
 * (Miller-Rabin), builds Y (a square root of −1 when p ≡ 1 mod 4, else
 * Y = I ⊗ [[a,b],[−b,a]] with a² + b² ≡ −1: Section 3.1, Prop. 3.2, Prop. 3.3,
 * Algorithm 3), chooses digits and chunk lengths, and allocates the
 * workspace (cudaMalloc).  On failure *plan is set to NULL. */
ffsyrk_status_t ffsyrk_plan(ffsyrk_plan_t *plan, uint32_t p, int64_t max_n, int64_t max_k,
                            const ffsyrk_options_t *opts);

/* Device memory a plan made by ffsyrk_plan with these arguments allocates at
 * creation, computed on the host (no GPU needed, for capacity planning):
 * *workspace_bytes = the plan's workspace (ffsyrk_plan_info_t's
 * workspace_bytes), *slot_bytes (may be NULL) = the partial-result slots of
 * shared tiles for a device with `sms` SMs (0: 152, GB300).  Buffers made on
 * first use are not included (the scaled products' Ā and planner table, the
 * host entry point's copies of A and C).  Same argument checks as
 * ffsyrk_plan. */
ffsyrk_status_t ffsyrk_workspace_query(uint32_t p, int64_t max_n, int64_t max_k,
                                       const ffsyrk_options_t *opts, int32_t sms,
                                       int64_t *workspace_bytes, int64_t *slot_bytes);

/* Free the plan's workspace.  Synchronises the device work it enqueued.
 * NULL is accepted. */
ffsyrk_status_t ffsyrk_plan_destroy(ffsyrk_plan_t plan);

/* C = A·Aᵀ mod p (triangle `uplo`) with an existing plan; p must equal the
 * plan's p and n ≤ max_n, k ≤ max_k. */
ffsyrk_status_t ffsyrk_with_plan(ffsyrk_plan_t plan, ffsyrk_uplo_t uplo, int64_t n, int64_t k,
                                 uint32_t p, const uint32_t *A, int64_t lda, uint32_t *C,
                                 int64_t ldc, ffsyrk_stream_t stream);

/* C = A·Aᵀ mod p for HOST matrices, with a plan: A (n × k, row stride lda)
 * is copied to device memory the plan owns (allocated on the first such call,
 * max_n × max_k and max_n × max_n uint32), the product runs there, and the
 * whole n × n result comes back to the host matrix C (row stride ldc): the
 * triangle `uplo` of A·Aᵀ mod p and zeros in the other strict triangle (one
 * contiguous copy when ldc = n: full-rate transfers, unlike copies of a
 * triangle's shorter rows).  Everything is enqueued on `stream`: the call
 * returns before the copies finish, and the host buffers must stay valid
 * until the stream has drained them (pinned host memory lets the copies
 * overlap other work; pageable memory works but copies synchronously).
 * Calls on one plan reuse its device buffers, so a pipeline of calls uses one
 * plan per call in flight. */
ffsyrk_status_t ffsyrk_host(ffsyrk_plan_t plan, ffsyrk_uplo_t uplo, int64_t n, int64_t k,
                            uint32_t p, const uint32_t *A, int64_t lda, uint32_t *C, int64_t ldc,
                            ffsyrk_stream_t stream);

/* C = A·Aᵀ mod p with default options, through an internal per-device plan
 * cache keyed by (p, shape): at most 8 plans, the least recently used one
 * released first.  If a new plan's workspace cannot be allocated, the cache
 * releases this device's plans (waiting for their work) and tries once more.
 * Thread-safe. */
ffsyrk_status_t ffsyrk(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p, const uint32_t *A,
                       int64_t lda, uint32_t *C, int64_t ldc, ffsyrk_stream_t stream);

/* The update C ← α·A·Aᵀ + β·C mod p (Section 4.2, Table 4: the general
 * operation whose schedule adds β·C into the blocks of the result).  Only the
 * triangle `uplo` of C is read and written; the other strict triangle is not
 * touched.  alpha and beta are any uint32 and are reduced mod p; α = 1,
 * β = 0 is the plain product (ffsyrk_with_plan).  The current contents of
 * C's triangle must be residues < p when β ≠ 0.  k = 0 gives C ← β·C.
 * Same plan, argument and error rules as ffsyrk_with_plan. */
ffsyrk_status_t ffsyrk_with_plan_update(ffsyrk_plan_t plan, ffsyrk_uplo_t uplo, int64_t n,
                                        int64_t k, uint32_t p, uint32_t alpha, const uint32_t *A,
                                        int64_t lda, uint32_t beta, uint32_t *C, int64_t ldc,
                                        ffsyrk_stream_t stream);

/* The same update through the internal plan cache (as ffsyrk).  Thread-safe. */
ffsyrk_status_t ffsyrk_update(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                              const uint32_t *A, int64_t lda, uint32_t beta, uint32_t *C,
                              int64_t ldc, ffsyrk_stream_t stream);

/* Symmetric product with diagonal scaling, C ← α·A·D·Aᵀ + β·C mod p with
 * D = Diag(d[0..k−1]) (Section 5, Algorithm 5 "syrkd"; for an LDLᵀ update
 * C ← C − A·D·Aᵀ take α = p − 1, β = 1).  d is a HOST array of k entries
 * (any uint32, reduced mod p).  D is factored as Δ·Δᵀ without field
 * extensions: a square root for each square d_j (0 included), the 2×2
 * matrix of Algorithm 4 ("nrsyf") for each pair of non-squares, and one extra
 * zero column of A when their number is odd; the scaled Ā = [A 0]·Δ goes
 * through the same path as ffsyrk_with_plan_update.  The plan must have
 * max_k ≥ k + 1 when d holds an odd number of non-squares
 * (FFSYRK_ERR_TOO_LARGE otherwise).  The first call needing more scratch than
 * the plan holds allocates it (cudaMalloc, after synchronising `stream`);
 * the column table is copied from pageable host memory.  Other rules as for
 * ffsyrk_with_plan_update. */
ffsyrk_status_t ffsyrkd_with_plan_update(ffsyrk_plan_t plan, ffsyrk_uplo_t uplo, int64_t n,
                                         int64_t k, uint32_t p, uint32_t alpha, const uint32_t *A,
                                         int64_t lda, const uint32_t *d, uint32_t beta, uint32_t *C,
                                         int64_t ldc, ffsyrk_stream_t stream);

/* The same through the internal plan cache (plans made with max_k = k + 1).
 * Thread-safe. */
ffsyrk_status_t ffsyrkd_update(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                               const uint32_t *A, int64_t lda, const uint32_t *d, uint32_t beta,
                               uint32_t *C, int64_t ldc, ffsyrk_stream_t stream);

/* The factorisation step of Algorithm 5 on the host (for tests and tools;
 * needs no GPU): for the k entries d, writes the column transform of
 * Ā = [A 0]·Δ -- column c of Ā is u[c]·Ā_c + v[c]·Ā_{partner[c]}, partner
 * −1 meaning none, Ā_c = 0 for c ≥ k -- into partner, u, v (each with room
 * for k + 1 entries).  Returns the column count of Ā (k or k + 1), or −1. */
int32_t ffsyrkd_factor(uint32_t p, int64_t k, const uint32_t *d, int32_t *partner, uint32_t *u,
                       uint32_t *v);

/* Symmetric product with block-diagonal scaling, C ← α·A·B·Aᵀ + β·C mod p
 * (Section 5, Algorithm 6 "syrkbd", odd characteristic), with B symmetric,
 * block diagonal with 1×1 and 2×2 blocks: d[0..k−1] is B's diagonal and
 * e[0..k−2] its first off-diagonal, B[j][j+1] = B[j+1][j] = e[j]; a nonzero
 * e[j] (mod p) opens the 2×2 block on columns j, j+1.  d and e are HOST
 * arrays (any uint32, reduced mod p); e may be NULL (B = Diag(d), the same
 * as ffsyrkd_with_plan_update).  Each block [[x, β], [β, γ]] is congruent to a
 * diagonal one: for x = γ = 0 by the paper's antidiagonal identity (columns
 * A_j ± A_{j+1}, diagonal ±β/2), otherwise by one elimination step; the
 * resulting diagonal then goes through Algorithm 5, so Ā has k or k + 1
 * columns.  FFSYRK_ERR_INVALID_ARG when two blocks overlap (e[j] and e[j+1]
 * both nonzero mod p).  Other rules as for ffsyrkd_with_plan_update. */
ffsyrk_status_t ffsyrkbd_with_plan_update(ffsyrk_plan_t plan, ffsyrk_uplo_t uplo, int64_t n,
                                          int64_t k, uint32_t p, uint32_t alpha,
                                          const uint32_t *A, int64_t lda, const uint32_t *d,
                                          const uint32_t *e, uint32_t beta, uint32_t *C,
                                          int64_t ldc, ffsyrk_stream_t stream);

/* The same through the internal plan cache (plans made with max_k = k + 1).
 * Thread-safe. */
ffsyrk_status_t ffsyrkbd_update(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p,
                                uint32_t alpha, const uint32_t *A, int64_t lda, const uint32_t *d,
                                const uint32_t *e, uint32_t beta, uint32_t *C, int64_t ldc,
                                ffsyrk_stream_t stream);

/* The planning step of Algorithm 6 (with Algorithm 5) on the host, needing no
 * GPU: writes Ā = A·W with A·B·Aᵀ = Ā·Āᵀ, column c of Ā being
 * Σ_{t<4} w[4c+t]·A_{src[4c+t]} (src −1: unused term; every src < k).  src
 * and w need room for 4·(k + 1) entries.  Returns the column count of Ā
 * (k or k + 1), or −1 for a bad p, bad sizes or overlapping blocks. */
int32_t ffsyrkbd_factor(uint32_t p, int64_t k, const uint32_t *d, const uint32_t *e, int32_t *src,
                        uint32_t *w);

/* The same planning step as ffsyrkbd_factor, run by the device planner that
 * ffsyrkbd_with_plan_update uses (on the current device, synchronously, with
 * its own temporary buffers): the two are meant to give the same W entry for
 * entry.  Returns the column count of Ā, −1 for bad arguments, −2 when a CUDA
 * call or a device-side check fails. */
int32_t ffsyrkbd_factor_device(uint32_t p, int64_t k, const uint32_t *d, const uint32_t *e,
                               int32_t *src, uint32_t *w);

/* ---- Hermitian product over F_{p²} (Section 3.2, "Conjugate transpose") ----
 *
 * C = A·Aᴴ for A ∈ F_{p²}^{n×k}, F_{p²} = F_p[i]/(i² − r) with r a non-square
 * mod p, conjugation x + y·i ↦ x − y·i (the Frobenius map).  A is stored
 * interleaved as an n × 2k uint32 matrix Z (row j: Re A[j][0], Im A[j][0],
 * Re A[j][1], …; row stride lda ≥ 2k, entries any uint32, reduced mod p).
 * The result goes to two n × n uint32 matrices (row stride ldc), the
 * triangle `uplo` of Re C (symmetric) and of Im C (antisymmetric, zero
 * diagonal); the other strict triangles are not touched.
 *
 * The paper runs Algorithm 2 over F_{p²} with a Y satisfying Y·Yᴴ = −I.
 * This library computes the same C through products over F_p:
 * Re C = Z·Diag(1, −r, 1, −r, …)·Zᵀ (Algorithm 2 on Z, plain when r = −1,
 * otherwise through the diagonal scaling of Algorithm 5) and
 * Im C = Z·(Z·Jᵀ)ᵀ with J = I ⊗ [[0, −1], [1, 0]], one triangular general
 * product on the classical leaf (its operand Z·Jᵀ is digit-split directly
 * from Z).  A plan holds one plan of each kind. */
typedef struct ffherk_plan_st *ffherk_plan_t;

/* A plan for n ≤ max_n, k ≤ max_k (k counts F_{p²} columns).  r must be a
 * non-square mod p (FFSYRK_ERR_INVALID_ARG otherwise), e.g. p − 1 when
 * p ≡ 3 (mod 4).  opts applies to the real part's plan (levels, leaf,
 * tile widths, Winograd); the imaginary part always runs at depth 0. */
ffsyrk_status_t ffherk_plan(ffherk_plan_t *plan, uint32_t p, uint32_t r, int64_t max_n,
                            int64_t max_k, const ffsyrk_options_t *opts);
ffsyrk_status_t ffherk_plan_destroy(ffherk_plan_t plan);
/* Re C and Im C (triangle uplo) on `stream`; asynchronous like
 * ffsyrk_with_plan.  Cre and Cim must not overlap each other or A. */
ffsyrk_status_t ffherk_with_plan(ffherk_plan_t plan, ffsyrk_uplo_t uplo, int64_t n, int64_t k,
                                 const uint32_t *A, int64_t lda, uint32_t *Cre, uint32_t *Cim,
                                 int64_t ldc, ffsyrk_stream_t stream);
/* ffsyrk_sync_status for both of the plan's parts. */
ffsyrk_status_t ffherk_sync_status(ffherk_plan_t plan, ffsyrk_stream_t stream);
/* The same through an internal cache of plans keyed by (device, p, r, n, k):
 * at most 4, released as in ffsyrk's cache.  Thread-safe. */
ffsyrk_status_t ffherk(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p, uint32_t r,
                       const uint32_t *A, int64_t lda, uint32_t *Cre, uint32_t *Cim, int64_t ldc,
                       ffsyrk_stream_t stream);

/* `count` independent products C_t = A_t·A_tᵀ mod p of uneven sizes n[t] × k[t],
 * all with the same p and uplo.  n, k, lda, ldc are HOST arrays of `count`
 * values; A and C are HOST arrays of `count` DEVICE pointers.  Problems with
 * n[t] = 0 are skipped.  Workspace comes from an internal per-device cache. */
ffsyrk_status_t ffsyrk_batched(ffsyrk_uplo_t uplo, int64_t count, const int64_t *n,
                               const int64_t *k, uint32_t p, const uint32_t *const *A,
                               const int64_t *lda, uint32_t *const *C, const int64_t *ldc,
                               ffsyrk_stream_t stream);

/* C = A·Aᵀ mod p (triangle `uplo`) without allocating any memory.
 *
 * The paper has no counterpart: this is a deployment variant of the
 * classical path (levels = 0, tensor-core leaf, one-SM tiles).  It is for
 * callers that must not allocate device memory at call time: applications
 * whose pool allocator owns all device memory, processes under a fixed
 * memory budget, or latency-critical code where cudaMalloc/cudaFree (which
 * can synchronise the device) are not acceptable.  It calls no cudaMalloc,
 * cudaFree or other allocating routine; its scratch is one array compiled
 * into the library (64 MiB of digit planes + 2 MiB of launch descriptors and
 * tile list) that every GPU which loads the library holds until the process
 * exits.  It copies nothing from host memory (its descriptors reach the GPU
 * as a kernel parameter), so a call does not wait for earlier work on
 * `stream`.
 *
 * Limits (FFSYRK_ERR_TOO_LARGE before anything is enqueued):
 *   - the digit planes of A must fit:
 *     D · roundup(n,256) · roundup(k,64) · 2 bytes ≤ 64 MiB, where D is the
 *     digit count of p (2 for p < 2^17, 3 above; e.g. n = k = 4096, D = 2);
 *   - the stored triangle must cover at most 130432 output tiles of
 *     128 × 256 (n ≤ 92288 for the lower triangle, whatever k).
 *
 * Set-up: the first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.
 *
 * Sharing: all calls on a device share the one array and every call
 * overwrites it, so calls whose GPU work overlaps (different streams, or
 * threads without ordering between them) race and may produce wrong
 * results.  Calls on one stream are ordered and safe.  A device-side bounded
 * wait that runs out is not reported by this entry point.
 *
 * Arguments, layout and results are those of ffsyrk(). */
ffsyrk_status_t ffsyrk_noalloc(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p,
                               const uint32_t *A, int64_t lda, uint32_t *C, int64_t ldc,
                               ffsyrk_stream_t stream);

/* Wait for the plan's enqueued work on `stream` and report any device-side
 * failure recorded since the last call (then clear it). */
ffsyrk_status_t ffsyrk_sync_status(ffsyrk_plan_t plan, ffsyrk_stream_t stream);

/* What a plan chose, for tests and reports. */
typedef struct {
    uint32_t p;
    int32_t y_form;      /* 0: scalar Y = i·I; 1: Y = I ⊗ [[a,b],[−b,a]]   */
    uint32_t y_a;        /* i (scalar form) or a                          */
    uint32_t y_b;        /* b (2×2 form), else 0                          */
    int32_t y_cost;      /* y of Thm 4.1: 1, 2 or 3                       */
    int32_t leaf;        /* ffsyrk_leaf_t actually used                   */
    int32_t levels;      /* recursion levels L for max_n × max_k          */
    int32_t digits;      /* D, signed digits per residue (ffsyrk_digit_base) */
    int32_t chunk_k[9];  /* K-chunk per digit pair (i*3+j), TC leaf       */
    int64_t workspace_bytes;
    int32_t tile_ctas;   /* 1 or 2: SMs per tensor-core leaf tile at max_n  */
    int32_t autotuned;   /* 1 if levels/tile_ctas came from the autotuner    */
    float tuned_ms;      /* the winning candidate's time per call, or 0      */
    int32_t winograd[6]; /* levels of Algorithm 1 for the general products of
                            depth d = 0..5 at max_n × max_k (0 beyond L − 1) */
    int32_t planes;      /* digit planes per leaf operand (D, or D(D+1)/2
                            with Karatsuba digit products)                  */
    int32_t products;    /* digit products per field multiply-add of the
                            leaf: D², or D(D+1)/2 with Karatsuba; 1 for the
                            int64 leaf                                       */
    int32_t epilogue_warps; /* one-SM tensor-core leaf: epilogue warps (8 or
                            16; 0 for the other leaves)                      */
    int32_t unit_bounds; /* the unit_bounds option the plan runs with       */
} ffsyrk_plan_info_t;

ffsyrk_status_t ffsyrk_plan_get_info(ffsyrk_plan_t plan, ffsyrk_plan_info_t *info);

/* Device timing of a plan's calls, for benchmarks and tracing.  While
 * enabled, every call records CUDA events on its stream before the first
 * launch, between the stage groups (pre-additions/digit split, leaf
 * products, post-additions) and after the last launch.  Enabling allocates
 * four events (cudaEventCreate). */
ffsyrk_status_t ffsyrk_plan_set_timing(ffsyrk_plan_t plan, int32_t enable);

typedef struct {
    float prep_ms;            /* pre-additions and digit split (Algorithm 2, S1..S4) */
    float leaf_ms;            /* the grouped leaf-product launch (P1..P5 leaves)      */
    float post_ms;            /* post-additions (U1..U5)                              */
    float total_ms;
    int32_t launches;         /* kernel launches of the call                          */
    int32_t leaf_launches;
    double field_macs;        /* useful multiply-adds mod p of the leaf products      */
    double tensor_macs;       /* digit-pair multiply-adds issued for them (D²×)       */
    int32_t leaf_tiles;       /* output tiles of the leaf launch                      */
    int32_t leaf_entries;     /* work entries handed to its CTAs                      */
    int32_t split_tiles;      /* tiles whose K schedule several CTAs share (a launch
                                 with few, long tiles: each CTA takes an equal share
                                 of the K units and the last to finish a tile adds
                                 the others' partial residues)                        */
    int32_t reserved;
} ffsyrk_timing_t;

/* Timing of the most recent call with timing enabled: waits for its last
 * event.  FFSYRK_ERR_INVALID_ARG if timing is off or no call was made. */
ffsyrk_status_t ffsyrk_plan_get_timing(ffsyrk_plan_t plan, ffsyrk_timing_t *timing);

/* Accumulator units of the most recent call's tensor-core leaf, summed over
 * its distinct K schedules (the delayed reduction of Section 4.2: one
 * reduction per unit): *host_units as the worst-case schedule has them,
 * *units as the leaf ran them (equal with unit_bounds = 1; with 0, after the
 * data-driven merge of that call).  Synchronises `stream` and reads the
 * schedule back from the device.  FFSYRK_ERR_INVALID_ARG if no tensor-core
 * call was made with the plan. */
ffsyrk_status_t ffsyrk_plan_units(ffsyrk_plan_t plan, ffsyrk_stream_t stream, int64_t *host_units,
                                  int64_t *units);

/* Throughput probe of an arithmetic pipe a leaf can use (the paper has no
 * counterpart; it measures the roofline denominators that no measured peak
 * on file covers).  Enqueues on `stream` one launch of `blocks` × 256
 * threads, each running `iters` rounds (≤ 2^24) of 8 independent
 * multiply-add chains on register operands:
 *   kind 0: mma.sync.m16n8k32 s8·s8 → s32;  1: u8·s8 → s32;  2: u8·u8 → s32;
 *   kind 3: mad.wide.u32 (32 × 32 → 64 bits, CUDA cores);
 *   kind 4: mma.sync.m16n8k16 bf16·bf16 → f32.
 * *macs receives the multiply-adds the launch performs (time it with events
 * on `stream`).  `sink` is a device word the kernel may xor into.  Invalid
 * arguments return FFSYRK_ERR_INVALID_ARG before any launch. */
ffsyrk_status_t ffsyrk_probe_pipe(int32_t kind, int64_t iters, int32_t blocks, uint32_t *sink,
                                  ffsyrk_stream_t stream, double *macs);

/* Failure-injection hook for tests (the paper has no counterpart): after
 * `skip` more successful device allocations of plan creation (a plan's
 * workspace and shared-tile slots), the next `count` such allocations fail
 * as if the device were out of memory, and ffsyrk_plan (or the plan cache
 * behind ffsyrk) sees FFSYRK_ERR_ALLOC.  count = 0 clears the hook.  Returns
 * the failures that were still pending.  Process-wide; nothing is enqueued. */
int32_t ffsyrk_test_inject_alloc_failure(int32_t skip, int32_t count);

/* The plan cache behind ffsyrk(), ffsyrk_update() and the scaled entry
 * points: *plans = the plans it holds for the current device; *releases =
 * how often (process-wide) a plan creation that failed with
 * FFSYRK_ERR_ALLOC made it release the device's cached plans and try once
 * more.  Either pointer may be NULL. */
ffsyrk_status_t ffsyrk_cache_info(int32_t *plans, int64_t *releases);

/* Failure-detection self-test (the paper has no counterpart): enqueue on
 * `stream` a kernel whose bounded device-side wait runs out after limit_ns
 * nanoseconds (≤ 10 s) on a barrier that nothing signals.  It records the
 * timeout in the plan exactly as a stalled leaf kernel would, and returns
 * normally: the next ffsyrk_sync_status() reports FFSYRK_ERR_TIMEOUT (and
 * clears it) and the plan and context remain usable. */
ffsyrk_status_t ffsyrk_plan_selftest_timeout(ffsyrk_plan_t plan, int64_t limit_ns,
                                             ffsyrk_stream_t stream);

/* Introspection of the tensor-core leaf's exact-accumulation schedule for p
 * and a leaf K of 64·kblocks (for tests and tools; needs no GPU).
 * Writes up to `cap` segments as 5 int32 each: digit i, digit j, first
 * k-block, k-block count, 1 if the segment opens a new FP32 accumulator
 * (unit).  Returns the number of segments, or −1 for a bad p or argument.
 * Every unit holds one weight class i + j and satisfies
 * Σ 64·count·bound(i)·bound(j) ≤ 2^24 with the bounds of
 * ffsyrk_digit_bounds(). */
int32_t ffsyrk_leaf_schedule(uint32_t p, int32_t kblocks, int32_t *out, int32_t cap);

/* The same with Karatsuba digit products (option digit_products = 2), for
 * a leaf K of 64·kblocks: every segment multiplies plane i of X by plane i
 * of Z (i = j in the output), planes as ffsyrk_digit_planes() lists them;
 * every unit holds one product and satisfies Σ 64·count·bound(i)² ≤ 2^24.
 * Returns −1 for a bad p or argument. */
int32_t ffsyrk_leaf_schedule_ks(uint32_t p, int32_t kblocks, int32_t *out, int32_t cap);

/* The Karatsuba digit planes of p: 0 if they do not apply (a digit sum
 * could exceed 256, or one digit), else the plane count P = D(D+1)/2 with
 * max_digit[t] the bound on plane t (planes 0..D−1 the digits of
 * ffsyrk_digit_bounds(), then the sums (0,1), (0,2), (1,2)) and weight[t]
 * the residue w_t with X·Zᵀ ≡ Σ_t w_t·plane_t(X)·plane_t(Z)ᵀ (mod p).
 * Arrays of 6 entries.  −1 for a bad p. */
int32_t ffsyrk_digit_planes(uint32_t p, int32_t *max_digit, uint32_t *weight);

/* The same for the INT8 leaf (FFSYRK_LEAF_I8), for a leaf K of
 * 128·kblocks: digits are the bytes of the two's-complement symmetric
 * residue (unsigned below the top digit, signed at the top); every unit
 * holds one weight class i + j and satisfies
 * Σ 128·count·bound(i)·bound(j) ≤ 2^30 with the bounds of
 * ffsyrk_i8_digit_bounds(). */
int32_t ffsyrk_i8_schedule(uint32_t p, int32_t kblocks, int32_t *out, int32_t cap);

/* The INT8 leaf's digit count of p (the least D whose top byte holds the
 * sign of every symmetric residue) and the bound on |digit t| (255 below
 * the top digit).  Returns D, or −1. */
int32_t ffsyrk_i8_digit_bounds(uint32_t p, int32_t *max_digit);

/* The signed digit count D of p and the bound on |digit t| for t < D
 * (written to max_digit[0..D−1]), for the digit base ffsyrk_digit_base(p).
 * Returns D, or −1. */
int32_t ffsyrk_digit_bounds(uint32_t p, int32_t *max_digit);

/* The base of the signed digits the tensor-core leaf splits residues into:
 * 256, except for two-digit primes above 2^16, where a balanced base b ≈ √p
 * keeps both digits within b/2 ≤ 256 (for p = 131071: 362).  Digits are
 * d_0 = s − b·round(s/b), d_1 = round(s/b) of the signed residue s.
 * Returns the base, or −1 for an unsupported p. */
int32_t ffsyrk_digit_base(uint32_t p);

/* Human-readable name of a status code (static storage). */
const char *ffsyrk_status_string(ffsyrk_status_t status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t ffsyrk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FFSYRK_H */
