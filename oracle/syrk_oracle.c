/*
 * Schoolbook oracle for C = A·Aᵀ mod p (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this file's library.  It shares no code, header, table or constant
 * with the CUDA path; it is the plain definition of the product that the
 * paper's Algorithm 2 reaches exactly (Section 3, "the lower left triangular
 * part of C = A·Aᵀ"; the SYRK terminology of Section 1):
 *
 *     C[i][j] = ( Σ_{l<k} (A[i][l] mod p) · (A[j][l] mod p) ) mod p.
 *
 * Every entry of A may be any uint32; A is reduced mod p first, entry by
 * entry, into a private copy (the input is never modified).  Each
 * product is < p² < 2^48 (p < 2^24), so a uint64 running sum is reduced
 * every 2^15 terms (2^15 · 2^48 = 2^63 < 2^64) and can never wrap.
 * Work is split over POSIX threads by output rows; the arithmetic of each
 * entry is independent of the split.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_REDUCE_EVERY 32768

/* One entry: the dot product of rows i and j of the reduced A, mod p.
 * Both rows already hold residues in [0, p). */
static uint32_t dot_mod_p(const uint32_t *ri, const uint32_t *rj, int64_t k, uint64_t p) {
    uint64_t acc = 0;
    int64_t since = 0;
    for (int64_t l = 0; l < k; ++l) {
        uint64_t a = ri[l];
        uint64_t b = rj[l];
        acc += a * b;
        if (++since == ORACLE_REDUCE_EVERY) {
            acc %= p;
            since = 0;
        }
    }
    return (uint32_t)(acc % p);
}

enum { JOB_LOWER = 0, JOB_UPPER = 1, JOB_FULL = 2, JOB_ROWS = 3 };

typedef struct {
    int kind;
    int64_t n, k;
    uint64_t p;
    const uint32_t *A;
    const uint32_t *B; /* the right-hand rows: A, or A with column l times d[l] */
    const uint32_t *d; /* NULL, or the diagonal of D for A·D·Aᵀ (of B for A·B·Aᵀ) */
    const uint32_t *e; /* NULL, or B's first off-diagonal: B[l][l+1] = B[l+1][l] = e[l] */
    int64_t lda;
    uint32_t *C;
    int64_t ldc;
    const int64_t *rows; /* JOB_ROWS: the sampled rows */
    int64_t nrows;
    int64_t t, nthreads;
} job_t;

static void *worker(void *arg) {
    const job_t *j = (const job_t *)arg;
    int64_t count = (j->kind == JOB_ROWS) ? j->nrows : j->n;
    /* cyclic split so that triangular rows balance */
    for (int64_t r = j->t; r < count; r += j->nthreads) {
        if (j->kind == JOB_ROWS) {
            int64_t i = j->rows[r];
            const uint32_t *ri = j->A + i * j->lda;
            uint32_t *out = j->C + r * j->ldc;
            for (int64_t c = 0; c < j->n; ++c)
                out[c] = dot_mod_p(ri, j->B + c * j->lda, j->k, j->p);
        } else {
            int64_t i = r;
            const uint32_t *ri = j->A + i * j->lda;
            int64_t c0 = 0, c1 = j->n; /* columns [c0, c1) of row i */
            if (j->kind == JOB_LOWER) c1 = i + 1;
            if (j->kind == JOB_UPPER) c0 = i;
            for (int64_t c = c0; c < c1; ++c)
                j->C[i * j->ldc + c] = dot_mod_p(ri, j->B + c * j->lda, j->k, j->p);
        }
    }
    return NULL;
}

/* A mod p, entry by entry, into a fresh n×k array (freed by the caller). */
static uint32_t *reduce_copy(int64_t n, int64_t k, uint64_t p, const uint32_t *A, int64_t lda) {
    size_t cnt = (size_t)(n > 0 ? n : 1) * (size_t)(k > 0 ? k : 1);
    uint32_t *R = (uint32_t *)malloc(cnt * sizeof(uint32_t));
    if (!R) return NULL;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t l = 0; l < k; ++l) R[i * k + l] = (uint32_t)((uint64_t)A[i * lda + l] % p);
    return R;
}

static int run(job_t proto, int nthreads) {
    uint32_t *R = reduce_copy(proto.n, proto.k, proto.p, proto.A, proto.lda);
    if (!R) return -1;
    /* with a diagonal: S[i][l] = R[i][l]·(d[l] mod p) mod p; with an
     * off-diagonal too, S = (A·B) mod p for the symmetric tridiagonal B:
     * S[i][l] = R[i][l]·d[l] + R[i][l−1]·e[l−1] + R[i][l+1]·e[l] (mod p) */
    uint32_t *S = NULL;
    if (proto.d) {
        const int64_t k = proto.k;
        const uint64_t p = proto.p;
        S = reduce_copy(proto.n, k, p, R, k > 0 ? k : 1);
        if (!S) {
            free(R);
            return -1;
        }
        for (int64_t i = 0; i < proto.n; ++i) {
            const uint32_t *ri = R + i * k;
            for (int64_t l = 0; l < k; ++l) {
                uint64_t s = (uint64_t)ri[l] * (proto.d[l] % p) % p;
                if (proto.e && l > 0) s += (uint64_t)ri[l - 1] * (proto.e[l - 1] % p) % p;
                if (proto.e && l + 1 < k) s += (uint64_t)ri[l + 1] * (proto.e[l] % p) % p;
                S[i * k + l] = (uint32_t)(s % p);
            }
        }
    }
    proto.A = R;
    proto.B = S ? S : R;
    proto.lda = proto.k > 0 ? proto.k : 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    if (!th || !jobs) {
        free(th);
        free(jobs);
        free(R);
        free(S);
        return -1;
    }
    int started = 0, rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].t = t;
        jobs[t].nthreads = nthreads;
        if (pthread_create(&th[t], NULL, worker, &jobs[t]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    /* threads that failed to start: finish their share here */
    for (int t = started; t < nthreads; ++t) worker(&jobs[t]);
    free(th);
    free(jobs);
    free(R);
    free(S);
    return rc < 0 && started == 0 ? -1 : 0;
}

/*
 * uplo 0: C[i][j] for j <= i (lower, diagonal included); uplo 1: j >= i
 * (upper); uplo 2: every entry, each computed on its own (never mirrored),
 * so that symmetry of the result is a real check.  Entries outside the
 * selected set are not written.  Returns 0, or -1 on bad arguments.
 */
int oracle_syrk_modp(int64_t n, int64_t k, uint32_t p, const uint32_t *A, int64_t lda,
                     uint32_t *C, int64_t ldc, int uplo, int nthreads) {
    if (n < 0 || k < 0 || p < 2 || lda < (k > 1 ? k : 1) || ldc < (n > 1 ? n : 1)) return -1;
    if (uplo < 0 || uplo > 2) return -1;
    if (n == 0) return 0;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = uplo == 0 ? JOB_LOWER : (uplo == 1 ? JOB_UPPER : JOB_FULL);
    j.n = n;
    j.k = k;
    j.p = p;
    j.A = A;
    j.lda = lda;
    j.C = C;
    j.ldc = ldc;
    return run(j, nthreads);
}

/*
 * Full rows of A·Aᵀ mod p for a sample of row indices: out[t][c] for
 * c < n is entry (rows[t], c).  out is nrows × ldo.  Used to check large
 * products one sampled row at a time.
 */
int oracle_syrk_rows(int64_t n, int64_t k, uint32_t p, const uint32_t *A, int64_t lda,
                     const int64_t *rows, int64_t nrows, uint32_t *out, int64_t ldo, int nthreads) {
    if (n < 0 || k < 0 || p < 2 || lda < (k > 1 ? k : 1) || ldo < (n > 1 ? n : 1) || nrows < 0)
        return -1;
    for (int64_t t = 0; t < nrows; ++t)
        if (rows[t] < 0 || rows[t] >= n) return -1;
    if (n == 0 || nrows == 0) return 0;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_ROWS;
    j.n = n;
    j.k = k;
    j.p = p;
    j.A = A;
    j.lda = lda;
    j.C = out;
    j.ldc = ldo;
    j.rows = rows;
    j.nrows = nrows;
    return run(j, nthreads);
}

/*
 * A·D·Aᵀ mod p with D = Diag(d[0..k-1]) (the product Algorithm 5, syrkd,
 * computes): C[i][j] = ( Σ_l (A[i][l] mod p)·(d[l] mod p)·(A[j][l] mod p) ) mod p,
 * on the triangle uplo (0 lower, 1 upper, 2 every entry).  The right-hand row
 * is scaled first, (A[j][l]·d[l]) mod p, so every product stays below p².
 */
int oracle_syrkd_modp(int64_t n, int64_t k, uint32_t p, const uint32_t *A, int64_t lda,
                      const uint32_t *d, uint32_t *C, int64_t ldc, int uplo, int nthreads) {
    if (n < 0 || k < 0 || p < 2 || lda < (k > 1 ? k : 1) || ldc < (n > 1 ? n : 1)) return -1;
    if (uplo < 0 || uplo > 2 || (k > 0 && !d)) return -1;
    if (n == 0) return 0;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = uplo == 0 ? JOB_LOWER : (uplo == 1 ? JOB_UPPER : JOB_FULL);
    j.n = n;
    j.k = k;
    j.p = p;
    j.A = A;
    j.d = d;
    j.lda = lda;
    j.C = C;
    j.ldc = ldc;
    return run(j, nthreads);
}

/*
 * A·B·Aᵀ mod p for a symmetric tridiagonal B given by its diagonal d[0..k-1]
 * and first off-diagonal e[0..k-2] (B[l][l+1] = B[l+1][l] = e[l]); this holds
 * the block-diagonal B of Algorithm 6 (syrkbd, Section 5), whose 2×2 blocks
 * sit on non-overlapping (l, l+1).  C[i][j] = Σ_l (A[i][l] mod p)·(A·B)[j][l]
 * mod p with (A·B)[j][l] reduced mod p first; e may be NULL (B diagonal).
 * Triangle uplo as above.  Returns 0, or -1 on bad arguments.
 */
int oracle_syrkbd_modp(int64_t n, int64_t k, uint32_t p, const uint32_t *A, int64_t lda,
                       const uint32_t *d, const uint32_t *e, uint32_t *C, int64_t ldc, int uplo,
                       int nthreads) {
    if (n < 0 || k < 0 || p < 2 || lda < (k > 1 ? k : 1) || ldc < (n > 1 ? n : 1)) return -1;
    if (uplo < 0 || uplo > 2 || (k > 0 && !d)) return -1;
    if (n == 0) return 0;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = uplo == 0 ? JOB_LOWER : (uplo == 1 ? JOB_UPPER : JOB_FULL);
    j.n = n;
    j.k = k;
    j.p = p;
    j.A = A;
    j.d = d;
    j.e = k > 1 ? e : NULL;
    j.lda = lda;
    j.C = C;
    j.ldc = ldc;
    return run(j, nthreads);
}

/*
 * Hermitian product over F_{p²} = F_p[i]/(i² − r), r a non-square mod p
 * (Section 3.2, "Conjugate transpose"): C = A·Aᴴ, C[j][l] = Σ_t A[j][t]·conj(A[l][t])
 * with conj(x + y·i) = x − y·i (the Frobenius map x ↦ x^p).  Written out:
 * (a + b·i)(c − d·i) = (ac − r·bd) + (bc − ad)·i.  A is interleaved: row j
 * holds Re A[j][0], Im A[j][0], Re A[j][1], ... (2k uint32, stride lda);
 * entries may be any uint32 (reduced mod p first).  Re C and Im C go to
 * Cre and Cim (stride ldc) on the triangle uplo (0 lower, 1 upper, 2 all).
 * Every term is reduced before it is added, so nothing can overflow.
 * Single-threaded (small cases only).  Returns 0, or -1 on bad arguments.
 */
int oracle_herk_modp(int64_t n, int64_t k, uint32_t p, uint32_t r, const uint32_t *A, int64_t lda,
                     uint32_t *Cre, uint32_t *Cim, int64_t ldc, int uplo) {
    if (n < 0 || k < 0 || p < 3 || lda < (2 * k > 1 ? 2 * k : 1) || ldc < (n > 1 ? n : 1)) return -1;
    if (uplo < 0 || uplo > 2) return -1;
    const uint64_t P = p, R = r % p;
    for (int64_t j = 0; j < n; ++j) {
        int64_t l0 = 0, l1 = n;
        if (uplo == 0) l1 = j + 1;
        if (uplo == 1) l0 = j;
        for (int64_t l = l0; l < l1; ++l) {
            uint64_t re = 0, im = 0;
            for (int64_t t = 0; t < k; ++t) {
                const uint64_t a = A[j * lda + 2 * t] % P, b = A[j * lda + 2 * t + 1] % P;
                const uint64_t c = A[l * lda + 2 * t] % P, d = A[l * lda + 2 * t + 1] % P;
                const uint64_t bd = b * d % P;
                re = (re + a * c % P + (P - R * bd % P)) % P;
                im = (im + b * c % P + (P - a * d % P)) % P;
            }
            Cre[j * ldc + l] = (uint32_t)re;
            Cim[j * ldc + l] = (uint32_t)im;
        }
    }
    return 0;
}
