// Shared definitions of the THC-RR-CCSD CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/thc.h"

namespace thc {

// Status carrier used inside the library; converted to thc_status at the ABI.
struct Err {
    thc_status code = THC_OK;
    std::string msg;
    bool ok() const { return code == THC_OK; }
};

#define THC_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            return ::thc::Err{e_ == cudaErrorMemoryAllocation ? THC_ERR_OOM    \
                                                              : THC_ERR_CUDA,  \
                              std::string(#call) + ": " +                      \
                                  cudaGetErrorString(e_)};                     \
        }                                                                      \
    } while (0)

#define THC_TRY(expr)                                                          \
    do {                                                                       \
        ::thc::Err e_ = (expr);                                                \
        if (!e_.ok()) return e_;                                               \
    } while (0)

// Debugging hooks, armed at each thc_init from the environment:
// THC_FAIL_ALLOC_AT=n makes the n-th device allocation of the library after
// that point fail with THC_ERR_OOM (failure injection; counted across
// threads); THC_POISON_WORKSPACE=1 fills every scratch buffer with NaN bytes
// at the end of initialisation, so that a read of scratch the path has not
// written shows up as a non-finite result; THC_DEBUG_PRODUCTS=1 reports on
// stderr every product of at least 3e7 flops that runs on the CUDA cores
// although a tensor-core path is enabled, with the reason.
void debug_arm_from_env();
bool debug_alloc_fails();
bool debug_poison();
bool debug_products();

// A strided view of a matrix: element (r, c) lives at p[r*rs + c*cs].
template <typename T>
struct View {
    const T* p;
    long long rs, cs;
    View t() const { return View{p, cs, rs}; }
};

template <typename T>
View<T> rowmajor(const T* p, long long ld) { return View<T>{p, ld, 1}; }

// One (batched) matrix product  C_b = alpha * A_b B_b + beta * C_b, with
// A_b = A + b*sAb etc.  With reduce = true every batch is summed into a
// single C (a long inner dimension running over the batch).
template <typename T>
struct Gemm {
    int M = 0, N = 0, K = 0, batch = 1;
    View<T> A{}, B{};
    long long sAb = 0, sBb = 0;
    T* C = nullptr;
    long long ldc = 0, sCb = 0;
    double alpha = 1.0, beta = 0.0;
    bool reduce = false;
    // Optional split-K workspace (partials are summed deterministically).
    T* ws = nullptr;
    size_t ws_elems = 0;
    int splits = 1;        // set by the launcher
};

// Number of kernels this library has launched (all threads, all contexts).
long long launches();
void count_launches(int n);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (device, kernel); thread-safe.  cudaFuncSetAttribute acts
// on the current device only, so a process that launches on several devices
// needs the opt-in on each of them.
cudaError_t smem_optin(const void* kernel, int bytes);
// Number of SMs of the current device (cached per device).
int device_sms();

cudaError_t gemm_simt(const Gemm<double>& g, cudaStream_t s);
cudaError_t gemm_simt(const Gemm<float>& g, cudaStream_t s);

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace thc
