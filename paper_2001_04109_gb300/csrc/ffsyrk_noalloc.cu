// ffsyrk_noalloc: the classical tensor-core product with no allocation at all.
//
// Some callers cannot allocate device memory when they call us: code that
// runs after an application has handed all device memory to its own pool
// allocator, processes under a hard memory budget that forbids new
// allocations once initialised, or real-time paths where a cudaMalloc (which
// may synchronise the device and take an unbounded time) is not acceptable.
// For them this entry point takes its scratch from one fixed array compiled
// into the library instead of a plan's workspace.
//
// What it computes is what ffsyrk_with_plan computes with levels = 0 and the
// tensor-core leaf: the digit split of A followed by one lower- (or upper-)
// tile leaf launch writing C.  It reuses those two kernels unchanged, with
// one-SM 128×256 tiles taken whole from the leaf's device work queue in
// bands of 8 tile rows (the planned path may instead use SM-pair tiles,
// taller bands for short K, Karatsuba digit products, or share long tiles
// among idle SMs; the result is the same).
//
// Nothing is copied from host memory: a one-block set-up kernel receives the
// launch descriptors (tensor map, digit-split job, product, K schedule) as
// its by-value parameter and writes them, the tile list and zeroed counters
// into the array.  So a call does not wait for earlier work on its stream
// and leaves no host buffer that a later call could change under it.
//
// The scratch array: every GPU that loads this library holds it until the
// process exits (64 MiB of digit planes plus 2 MiB for the descriptors and
// the tile list).  All calls on a device share it and each call overwrites
// it, so calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race with each other.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/ffsyrk.h"
#include "ffsyrk_internal.h"
#include "field_host.h"

using namespace fsk;

namespace {

constexpr size_t kPlaneBytes = size_t(64) << 20;   // digit planes of A
constexpr size_t kHeaderBytes = size_t(2) << 20;   // descriptors, counters, tile list

// The scratch itself.  Host code must not use this name as an address: it
// is a host-side stand-in.  Host code uses the address cudaGetSymbolAddress
// returns for the current device (see device_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes + kPlaneBytes];

// Header layout inside the scratch (byte offsets).
constexpr size_t kErrOff = 0;      // device-side error word of the leaf kernel
constexpr size_t kCtrOff = 64;     // the leaf's work-queue counter
constexpr size_t kTmapOff = 256;   // one CUtensorMap (128 B, 64-B aligned)
constexpr size_t kJobOff = 512;    // one DigitizeJob
constexpr size_t kProdOff = 1024;  // one LeafProd
constexpr size_t kSegOff = 2048;   // the K schedule (LeafSeg table)
// The longest K schedule of any shape within the plane limit is 512
// segments (p = 509 or 131071 at the longest k); the parameter holds twice that.
constexpr int kMaxSegs = 1024;
constexpr size_t kTileOff = kSegOff + kMaxSegs * sizeof(LeafSeg);  // the tile list
constexpr int64_t kMaxTiles = (int64_t)((kHeaderBytes - kTileOff) / sizeof(LeafTile));
constexpr int kBandRows = 8;  // tile rows per band (the planned path's band for long K)

struct DeviceState {
    bool ready;
    unsigned char *scratch;  // device address of g_noalloc_scratch on that device
    int sms;
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// First call on a device (with that device current): resolve the array's
// device address.  Returns nullptr if the runtime cannot give it.
DeviceState *device_scratch(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return nullptr;
        }
        d.scratch = static_cast<unsigned char *>(ptr);
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        d.ready = true;
    }
    return &d;
}

inline int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Everything the set-up kernel writes, passed by value (about 9 KB).
struct SetupArgs {
    CUtensorMap tmap;
    DigitizeJob job;
    LeafProd prod;
    int32_t nseg;
    int32_t TM, TN;      // tile grid of the n × n output
    int32_t BM, BN;      // tile shape
    int32_t cost;        // per-tile cost recorded in the tile list
    LeafSeg segs[kMaxSegs];
};

// Tile (a, b) holds an entry of the stored triangle (tri 1: c ≤ r; 2: c ≥ r).
__host__ __device__ inline bool tile_live(int64_t a, int64_t b, int64_t n, int64_t BM, int64_t BN,
                                          int tri) {
    const int64_t r0 = a * BM, r1 = (r0 + BM < n ? r0 + BM : n) - 1;
    const int64_t c0 = b * BN, c1 = (c0 + BN < n ? c0 + BN : n) - 1;
    if (tri == 1 && r1 < c0) return false;
    if (tri == 2 && c1 < r0) return false;
    return true;
}

// Live tiles of one (band, column) item of the band order.
__host__ __device__ inline int item_tiles(int64_t item, int64_t TM, int64_t TN, int64_t n,
                                          int64_t BM, int64_t BN, int tri) {
    const int64_t band = item / TN, b = item % TN;
    const int64_t a0 = band * kBandRows, a1 = a0 + kBandRows < TM ? a0 + kBandRows : TM;
    int c = 0;
    for (int64_t a = a0; a < a1; ++a) c += tile_live(a, b, n, BM, BN, tri) ? 1 : 0;
    return c;
}

// One block: copy the descriptors, zero the counters, and list the live
// tiles in band order (bands of kBandRows tile rows, column by column inside
// a band, rows in order), the planned path's order for long-K products.
constexpr int kSetupThreads = 1024;
__global__ void __launch_bounds__(kSetupThreads) k_noalloc_setup(const __grid_constant__ SetupArgs a,
                                                                  unsigned char *hdr) {
    __shared__ int64_t part[kSetupThreads];
    const int t = threadIdx.x;
    // descriptors (8-byte words; every block's size is a multiple of 8)
    auto copy8 = [&](void *dst, const void *src, size_t bytes) {
        uint64_t *d = static_cast<uint64_t *>(dst);
        const uint64_t *s = static_cast<const uint64_t *>(src);
        for (size_t i = t; i < bytes / 8; i += kSetupThreads) d[i] = s[i];
    };
    static_assert(sizeof(CUtensorMap) % 8 == 0 && sizeof(DigitizeJob) % 8 == 0 &&
                      sizeof(LeafProd) % 8 == 0 && sizeof(LeafSeg) == 8,
                  "8-byte copies");
    copy8(hdr + kTmapOff, &a.tmap, sizeof(CUtensorMap));
    copy8(hdr + kJobOff, &a.job, sizeof(DigitizeJob));
    copy8(hdr + kProdOff, &a.prod, sizeof(LeafProd));
    copy8(hdr + kSegOff, a.segs, (size_t)a.nseg * sizeof(LeafSeg));
    if (t == 0) {
        *reinterpret_cast<unsigned int *>(hdr + kErrOff) = 0u;
        *reinterpret_cast<unsigned int *>(hdr + kCtrOff) = 0u;
    }
    // tile list: each thread takes a contiguous run of (band, column) items,
    // counts its tiles, and after an exclusive scan over the threads writes them
    const int64_t TM = a.TM, TN = a.TN, n = a.prod.rows;
    const int tri = a.prod.tri;
    const int64_t items = ((TM + kBandRows - 1) / kBandRows) * TN;
    const int64_t per = (items + kSetupThreads - 1) / kSetupThreads;
    const int64_t i0 = (int64_t)t * per, i1 = i0 + per < items ? i0 + per : items;
    int64_t cnt = 0;
    for (int64_t i = i0; i < i1; ++i) cnt += item_tiles(i, TM, TN, n, a.BM, a.BN, tri);
    part[t] = cnt;
    __syncthreads();
    for (int s = 1; s < kSetupThreads; s <<= 1) {  // inclusive scan (Hillis-Steele)
        const int64_t v = t >= s ? part[t - s] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t o = part[t] - cnt;
    LeafTile *tiles = reinterpret_cast<LeafTile *>(hdr + kTileOff);
    for (int64_t i = i0; i < i1; ++i) {
        const int64_t band = i / TN, b = i % TN;
        const int64_t a0 = band * kBandRows, a1 = a0 + kBandRows < TM ? a0 + kBandRows : TM;
        for (int64_t r = a0; r < a1; ++r)
            if (tile_live(r, b, n, a.BM, a.BN, tri)) tiles[o++] = LeafTile{0, (int32_t)r, (int32_t)b, a.cost};
    }
    // the leaf kernel reads the tensor map through the tensor-map proxy
    asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

}  // namespace

extern "C" ffsyrk_status_t ffsyrk_noalloc(ffsyrk_uplo_t uplo, int64_t n, int64_t k, uint32_t p,
                                          const uint32_t *A, int64_t lda, uint32_t *C,
                                          int64_t ldc, ffsyrk_stream_t stream) {
    if (p < 3 || p >= (1u << 24)) return FFSYRK_ERR_UNSUPPORTED_P;
    if (!host::is_prime(p)) return FFSYRK_ERR_NOT_PRIME;
    if (uplo != FFSYRK_LOWER && uplo != FFSYRK_UPPER) return FFSYRK_ERR_INVALID_ARG;
    if (n < 0 || k < 0) return FFSYRK_ERR_INVALID_ARG;
    if (lda < (k > 1 ? k : 1) || ldc < (n > 1 ? n : 1)) return FFSYRK_ERR_INVALID_ARG;
    if (n > 0 && (C == nullptr || (k > 0 && A == nullptr))) return FFSYRK_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) return FFSYRK_SUCCESS;
    if (k == 0)
        return launch_zero_tri(C, n, ldc, uplo == FFSYRK_UPPER, st) == cudaSuccess
                   ? FFSYRK_SUCCESS
                   : FFSYRK_ERR_CUDA;

    const DigitScheme ds = digit_scheme_for(p);
    const int64_t rpad = rup(n, 256), kpad = rup(k, 64);
    const int64_t BM = leaf_tc_bm(), BN = leaf_tc_bn();
    const int tri = uplo == FFSYRK_UPPER ? 2 : 1;
    // size limits: the digit planes must fit the array, and the triangle's
    // tiles the tile list
    if ((double)ds.D * (double)rpad * (double)kpad * 2.0 > (double)kPlaneBytes)
        return FFSYRK_ERR_TOO_LARGE;
    const int64_t TM = (n + BM - 1) / BM, TN = (n + BN - 1) / BN;
    if (TM > INT32_MAX || TN > INT32_MAX) return FFSYRK_ERR_TOO_LARGE;
    int64_t nt = 0;
    for (int64_t a = 0; a < TM; ++a)
        for (int64_t b = 0; b < TN; ++b) nt += tile_live(a, b, n, BM, BN, tri) ? 1 : 0;
    if (nt > kMaxTiles) return FFSYRK_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFSYRK_ERR_CUDA;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return FFSYRK_ERR_ARCH;

    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *ds_dev = device_scratch(dev);
    if (!ds_dev) return FFSYRK_ERR_CUDA;
    unsigned char *hdr = ds_dev->scratch;
    unsigned char *planes = ds_dev->scratch + kHeaderBytes;

    const ModP mp = make_modp(p, ds);

    Arena ar;
    ar.base = planes;
    ar.kind = ARENA_BF16;
    ar.planes = ds.D;
    ar.rpad = rpad;
    ar.kpad = kpad;
    ar.rows = ds.D * rpad;

    // the descriptors, written into the array by the set-up kernel
    static SetupArgs sa;  // ~9 KB; g_mu is held while it is filled and launched
    memset(&sa, 0, sizeof sa);
    if (!encode_arena_tmap(ar, &sa.tmap)) return FFSYRK_ERR_CUDA;
    sa.job.X = MatView{A, lda, n, k};
    sa.job.rows = n;
    sa.job.dst = OperandDst{planes, 0, kpad, rpad};
    LeafProd &pr = sa.prod;
    pr.arena = 0;
    pr.tri = tri;
    pr.a_row0 = pr.b_row0 = 0;
    pr.rows = pr.cols = n;
    pr.kblocks = (int32_t)(kpad / 64);
    pr.plane_rows = rpad;
    pr.out = C;
    pr.ldo = ldc;
    const int nseg = build_segments_into(ds, pr.kblocks, sa.segs, kMaxSegs);
    if (nseg < 0) return FFSYRK_ERR_TOO_LARGE;
    pr.seg0 = 0;
    pr.nseg = nseg;
    sa.nseg = nseg;
    sa.TM = (int32_t)TM;
    sa.TN = (int32_t)TN;
    sa.BM = (int32_t)BM;
    sa.BN = (int32_t)BN;
    sa.cost = pr.kblocks * ds.D * ds.D;

    k_noalloc_setup<<<1, kSetupThreads, 0, st>>>(sa, hdr);
    if (cudaGetLastError() != cudaSuccess) return FFSYRK_ERR_CUDA;
    cudaError_t e = launch_digitize(reinterpret_cast<const DigitizeJob *>(hdr + kJobOff), 1, n,
                                    kpad, mp, ds, ARENA_BF16, st);
    if (e != cudaSuccess) return FFSYRK_ERR_CUDA;
    TcLaunch tl{};
    tl.prods = reinterpret_cast<const LeafProd *>(hdr + kProdOff);
    tl.tiles = reinterpret_cast<const LeafTile *>(hdr + kTileOff);
    tl.segs = reinterpret_cast<const LeafSeg *>(hdr + kSegOff);
    tl.ntiles = (int)nt;
    tl.max_units = count_units(sa.segs, nseg);
    tl.tmaps = hdr + kTmapOff;
    tl.mp = mp;
    tl.ds = ds;
    tl.err = reinterpret_cast<unsigned int *>(hdr + kErrOff);
    tl.tile_ctr = reinterpret_cast<unsigned int *>(hdr + kCtrOff);
    e = launch_leaf_tc(tl, ds_dev->sms, st);
    return e == cudaSuccess ? FFSYRK_SUCCESS : FFSYRK_ERR_CUDA;
}
