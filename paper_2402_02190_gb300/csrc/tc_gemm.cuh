// Tensor-core (tcgen05 + TMA) dense layers for the BF16 form.
#pragma once

#include <string>

#include "kernels.cuh"

namespace cpra {

// True when this build carries the sm_103a tensor-core kernels.
bool tc_available();
// One-time host set-up (driver entry points, kernel attributes).
bool tc_prepare(int num_sms, std::string* msg);
// Whether a K-major x K-major product with this epilogue runs on tensor cores.
bool tc_gemm_supported(const GemmArgs& g);
// Launches it; returns the number of kernels launched.
int tc_gemm_launch(const GemmArgs& g, int num_sms, cudaStream_t st);
// FP32 operands to FP32 accuracy on the tensor cores (split TF32: B carries
// its hi part, B_lo its lo part, both K-major).
bool tc3_gemm_supported(const GemmArgs& g);
int tc3_gemm_launch(const GemmArgs& g, int num_sms, cudaStream_t st);
// Weight gradients (MN-major operands, split-K over the node dimension).
bool tc_wgrad_supported(const GemmArgs& g);
int tc_wgrad_launch(const GemmArgs& g, int num_sms, size_t part_floats, float* dst,
                    int64_t ldo, cudaStream_t st);

}  // namespace cpra
