// FP32 instantiations of the CUDA-core translate-product kernels (see k_gain_simt.cuh).
#include "k_gain_simt.cuh"

namespace dgfs {

namespace {
template <int NF>
cudaError_t dispatch_gp(const DevTables<float>& t, const float* f, const float* g, const int64_t* offs,
                        int64_t nodes, float* P, cudaStream_t s) {
    switch (t.N) {
        case 8: return simt::launch_gp<8, float, NF>(t, f, g, offs, nodes, P, s);
        case 16: return simt::launch_gp<16, float, NF>(t, f, g, offs, nodes, P, s);
        case 24: return simt::launch_gp<24, float, NF>(t, f, g, offs, nodes, P, s);
        case 32: return simt::launch_gp<32, float, NF>(t, f, g, offs, nodes, P, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_gain_products(const DevTables<float>& t, const float* f, const float* g,
                                      const int64_t* offs, int64_t nodes, float* P, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    return g ? dispatch_gp<2>(t, f, g, offs, nodes, P, s) : dispatch_gp<1>(t, f, nullptr, offs, nodes, P, s);
}


}  // namespace dgfs
