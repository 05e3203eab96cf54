// tcgen05 / TMA tile kernels (FP32 split, BF16, FP8).  Not available yet.
#include <cuda_runtime.h>

#include "abx_internal.h"

namespace abx {

bool umma_supported(int) { return false; }

cudaError_t launch_tile_umma(const TileGemmArgs &, int, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace abx
