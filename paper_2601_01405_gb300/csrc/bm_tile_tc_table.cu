// bm_tile_tc_table.cu -- table-mode instantiations of the tensor-core distance tiles (the
// inverted-file scan: work items read from a device table), compiled apart from the dense
// ones so that the two sets build in parallel.
#include "bm_tile_tc_kernel.cuh"

namespace bm {
namespace tc {

cudaError_t dispatch_table(const TileConfig& cfg, bool fp16, bool whole, TcArgs& args, long long a_rows_max,
                           cudaStream_t stream, std::string* why, int* grid_out) {
    return dispatch<true>(cfg, fp16, whole, args, a_rows_max, stream, why, grid_out);
}

}  // namespace tc
}  // namespace bm
