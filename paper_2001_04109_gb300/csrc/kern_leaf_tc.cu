// Tensor-core leaf (placeholder until the tcgen05 kernel lands).
#include "ffsyrk_internal.h"
namespace fsk {
int leaf_tc_bm() { return 128; }
int leaf_tc_bn() { return 256; }
cudaError_t launch_leaf_tc(const TcLaunch &, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace fsk
