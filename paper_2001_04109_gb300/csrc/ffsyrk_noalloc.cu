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
// What it computes is exactly what ffsyrk_with_plan computes with
// levels = 0 and the tensor-core leaf: the digit split of A followed by one
// lower- (or upper-) tile leaf launch writing C.  It reuses those two
// kernels unchanged; only the place their scratch lives differs.
//
// The scratch array: every GPU that loads this library holds it until the
// process exits (64 MiB of digit planes plus 1 MiB for the launch
// descriptors).  All calls on a device share it and each call overwrites
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
constexpr size_t kHeaderBytes = size_t(1) << 20;   // descriptors, tensor map, error word
constexpr int kMaxDevices = 64;

// The scratch itself.  Host code must not use this name as an address: it
// is a host-side stand-in.  Host code uses the address cudaGetSymbolAddress
// returns for the current device (see device_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes + kPlaneBytes];

struct DeviceState {
    bool ready;
    unsigned char *scratch;  // device address of g_noalloc_scratch on that device
    int sms;
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;
// host copy of the descriptor header; pageable, so cudaMemcpyAsync has
// staged it before returning and the next call may overwrite it
alignas(128) unsigned char g_stage[kHeaderBytes];

// Header layout inside the scratch (byte offsets).
constexpr size_t kErrOff = 0;      // device-side error word of the leaf kernel
constexpr size_t kTmapOff = 256;   // one CUtensorMap (128 B, 64-B aligned)
constexpr size_t kJobOff = 512;    // one DigitizeJob
constexpr size_t kProdOff = 1024;  // one LeafProd
constexpr size_t kSegOff = 2048;   // the K schedule (LeafSeg table)
constexpr size_t kMaxSegs = 8192;
constexpr size_t kTileOff = kSegOff + kMaxSegs * sizeof(LeafSeg);  // the tile list
constexpr size_t kMaxTiles = (kHeaderBytes - kTileOff) / sizeof(LeafTile);

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
    // size limits: the digit planes and the tile list must fit the array
    if ((double)ds.D * (double)rpad * (double)kpad * 2.0 > (double)kPlaneBytes)
        return FFSYRK_ERR_TOO_LARGE;
    const int64_t TM = (n + BM - 1) / BM, TN = (n + BN - 1) / BN;
    if (TM * TN > (int64_t)kMaxTiles || kpad / 64 > INT32_MAX) return FFSYRK_ERR_TOO_LARGE;

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

    Arena a;
    a.base = planes;
    a.kind = ARENA_BF16;
    a.planes = ds.D;
    a.rpad = rpad;
    a.kpad = kpad;
    a.rows = ds.D * rpad;

    // build the header on the host: error word zero, tensor map, job, product,
    // K schedule, tiles
    memset(g_stage, 0, kTileOff);
    if (!encode_arena_tmap(a, g_stage + kTmapOff)) return FFSYRK_ERR_CUDA;
    DigitizeJob job{};
    job.X = MatView{A, lda, n, k};
    job.rows = n;
    job.dst = OperandDst{planes, 0, kpad, rpad};
    memcpy(g_stage + kJobOff, &job, sizeof job);
    LeafProd pr{};
    pr.arena = 0;
    pr.tri = uplo == FFSYRK_UPPER ? 2 : 1;
    pr.a_row0 = pr.b_row0 = 0;
    pr.rows = pr.cols = n;
    pr.kblocks = (int32_t)(kpad / 64);
    pr.plane_rows = rpad;
    pr.out = C;
    pr.ldo = ldc;
    const int nseg = build_segments_into(ds, pr.kblocks,
                                         reinterpret_cast<LeafSeg *>(g_stage + kSegOff), (int)kMaxSegs);
    if (nseg < 0) return FFSYRK_ERR_TOO_LARGE;
    pr.seg0 = 0;
    pr.nseg = nseg;
    memcpy(g_stage + kProdOff, &pr, sizeof pr);
    int64_t nt = 0;
    LeafTile *tiles = reinterpret_cast<LeafTile *>(g_stage + kTileOff);
    for (int64_t tm = 0; tm < TM; ++tm)
        for (int64_t tn = 0; tn < TN; ++tn) {
            const int64_t r0 = tm * BM, r1 = (r0 + BM < n ? r0 + BM : n) - 1;
            const int64_t c0 = tn * BN, c1 = (c0 + BN < n ? c0 + BN : n) - 1;
            if (pr.tri == 1 && r1 < c0) continue;
            if (pr.tri == 2 && c1 < r0) continue;
            tiles[nt++] = LeafTile{0, (int32_t)tm, (int32_t)tn, pr.kblocks};
        }
    const size_t bytes = kTileOff + (size_t)nt * sizeof(LeafTile);
    if (cudaMemcpyAsync(hdr, g_stage, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FFSYRK_ERR_CUDA;

    cudaError_t e = launch_digitize(reinterpret_cast<const DigitizeJob *>(hdr + kJobOff), 1, n,
                                    kpad, mp, ds, ARENA_BF16, st);
    if (e != cudaSuccess) return FFSYRK_ERR_CUDA;
    TcLaunch tl{};
    tl.prods = reinterpret_cast<const LeafProd *>(hdr + kProdOff);
    tl.tiles = reinterpret_cast<const LeafTile *>(hdr + kTileOff);
    tl.segs = reinterpret_cast<const LeafSeg *>(hdr + kSegOff);
    tl.ntiles = (int)nt;
    tl.max_units = count_units(reinterpret_cast<const LeafSeg *>(g_stage + kSegOff), nseg);
    tl.tmaps = hdr + kTmapOff;
    tl.mp = mp;
    tl.ds = ds;
    tl.err = reinterpret_cast<unsigned int *>(hdr + kErrOff);
    tl.tile_ctr = nullptr;
    e = launch_leaf_tc(tl, ds_dev->sms, st);
    return e == cudaSuccess ? FFSYRK_SUCCESS : FFSYRK_ERR_CUDA;
}
