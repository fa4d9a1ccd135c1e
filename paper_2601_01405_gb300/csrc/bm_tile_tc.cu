// bm_tile_tc.cu -- K(b): tcgen05 tensor-core distance tiles (written next).
#include "bm_host.h"

namespace bm {

bool tc_supported() { return false; }

cudaError_t launch_sweep_tc(const SweepDesc&, cudaStream_t, std::string* why) {
    if (why) *why = "tensor-core tiles not built in this version";
    return cudaErrorNotSupported;
}

}  // namespace bm
