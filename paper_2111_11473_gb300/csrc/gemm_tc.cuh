// Tensor-core (tcgen05, bf16 hi/lo split) matrix product for float32 data.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace thc {

struct TcWorkspace {
    __nv_bfloat16* buf = nullptr;   // packed operands
    size_t elems = 0;
    float* partial = nullptr;       // split-K partial sums
    size_t partial_elems = 0;
    int* err = nullptr;             // set to 1 by a kernel whose bounded wait expired
};

// Packed-operand elements one product of this shape needs (upper bound).
size_t gemm_tc_pack_elems(int M, int N, int K, int batch, bool reduce);

// C = alpha op(A) op(B) + beta C on the tensor cores; nprod = 3 runs
// hi*hi + hi*lo + lo*hi, nprod = 1 runs hi*hi only.  Returns
// cudaErrorMemoryAllocation (without launching) if the workspace is too small.
cudaError_t gemm_tc(const Gemm<float>& g, const TcWorkspace& ws, int nprod, cudaStream_t s);

}  // namespace thc
