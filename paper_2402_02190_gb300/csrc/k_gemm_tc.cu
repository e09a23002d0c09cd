// Tensor-core dense layers (tcgen05 + TMA): not yet enabled in this build;
// every dense layer runs on the CUDA-core kernel.
#include "tc_gemm.cuh"

namespace cpra {

bool tc_available() { return false; }
bool tc_prepare(int, std::string* msg) {
  if (msg) *msg = "tensor-core path not built";
  return false;
}
bool tc_gemm_supported(const GemmArgs&) { return false; }
int tc_gemm_launch(const GemmArgs&, int, cudaStream_t) { return 0; }
bool tc_wgrad_supported(const GemmArgs&) { return false; }
int tc_wgrad_launch(const GemmArgs&, int, size_t, float*, int64_t, cudaStream_t) { return 0; }

}  // namespace cpra
