// Tensor-core translate-product path (16-bit precisions). Not built yet: every 16-bit
// precision reports DGFS_ERR_UNSUPPORTED at plan creation.
#include "tc_gain.h"

namespace dgfs {

bool tc_supported(int) { return false; }

int tc_extra_launches(int) { return 0; }

size_t build_tc_tables(const HostPlan&, int, std::vector<unsigned char>& blob, TcTables&) {
    blob.clear();
    return 0;
}

void rebase_tc_tables(TcTables&, void*) {}

cudaError_t launch_tc_gain_products(const TcTables&, int, const float*, const float*, const int64_t*,
                                    int64_t, float*, int*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace dgfs
