// placeholder until the tcgen05 path lands
#include "kernels.cuh"
namespace tatrg {
bool tc_available() { return false; }
void gemm_tc(const GemmDesc&, const double*, const double*, double*, int, cudaStream_t, Stats*) {
  throw Error(TATRG_ENOTIMPL, "tensor-core path not built");
}
}  // namespace tatrg
