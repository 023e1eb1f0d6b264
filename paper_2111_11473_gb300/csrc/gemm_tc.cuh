// Tensor-core (tcgen05, bf16 hi/lo split) matrix product for float32 data.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace thc {

struct TcWorkspace {
    __nv_bfloat16* buf = nullptr;   // packed operands
    size_t elems = 0;
    float* partial = nullptr;       // split-K partial sums
    size_t partial_elems = 0;
    int* err = nullptr;             // set to 1 by a kernel whose bounded wait expired
};

// Packed operands of buffers whose contents do not change (the inputs and
// the intermediates formed once at init): each distinct (buffer, view,
// shape) is packed on first use and reused afterwards.
struct PackCache {
    struct Range {
        const float* lo;
        const float* hi;
    };
    struct Entry {
        const float* p;
        long long rs, cs, bs;
        int R, Kd, nb, Rp, Kp, reduce, nprod;
        __nv_bfloat16* hi;
        __nv_bfloat16* lo;
    };
    std::vector<Range> constant;   // registered [lo, hi) address ranges
    std::vector<Entry> entries;
    size_t bytes = 0;
    size_t budget = 8ull << 30;    // packed bytes kept at most
    void add_constant(const float* p, size_t n) { constant.push_back({p, p + n}); }
    bool is_constant(const float* p) const {
        for (const Range& r : constant)
            if (p >= r.lo && p < r.hi) return true;
        return false;
    }
    // True if this operand is (or, within the budget, will be) cached.
    bool serves(const float* p, size_t packed_bytes, long long rs, long long cs, long long bs,
                int R, int Kd, int nb, int Rp, int Kp, int reduce, int nprod) const {
        if (!is_constant(p)) return false;
        for (const Entry& e : entries)
            if (e.p == p && e.rs == rs && e.cs == cs && e.bs == bs && e.R == R && e.Kd == Kd &&
                e.nb == nb && e.Rp == Rp && e.Kp == Kp && e.reduce == reduce && e.nprod == nprod)
                return true;
        return bytes + packed_bytes <= budget;
    }
    void release();
};

// Randomised comparison of gemm_tc with gemm_simt on the same float32 data:
// `cases` random shapes (M, N <= 700, K <= 900, batch <= 4), orientations,
// batch modes, beta and product counts.  *max_rel = the largest bf16x3
// difference relative to max(1, max |C|); *failures counts cases outside
// the arithmetic's bound (or with an expired wait).
cudaError_t gemm_tc_selftest(int cases, unsigned long long seed, double* max_rel, int* failures,
                             cudaStream_t st);

// Launch a single bounded wait on an mbarrier that is completed only if
// `complete` is non-zero; *flag (device) is set to 1 if the wait expired
// after `cycles` SM clocks.
cudaError_t wait_selftest(int complete, long long cycles, int* flag, cudaStream_t s);

// Packed-operand elements one product of this shape needs (upper bound).
size_t gemm_tc_pack_elems(int M, int N, int K, int batch, bool reduce);

// C = alpha op(A) op(B) + beta C on the tensor cores; nprod = 3 runs
// hi*hi + hi*lo + lo*hi, nprod = 1 runs hi*hi only.  Returns
// cudaErrorMemoryAllocation (without launching) if the workspace is too small.
cudaError_t gemm_tc(const Gemm<float>& g, const TcWorkspace& ws, int nprod, cudaStream_t s,
                    PackCache* cache = nullptr);

// Float64 products on the tensor cores: each operand row is cut into 8
// slices of 7-bit integers below a per-row power of two, the 36 slice pairs
// that matter are multiplied exactly (bf16 integer products, float32 sums of
// at most 1024 terms) and combined in float64, all in one fused kernel per
// product.  A product whose slices do not fit the workspace is cut into
// pieces that do; cudaErrorMemoryAllocation (without launching) only if a
// single 128 x 128 piece does not fit.
struct F64TcWorkspace {
    __nv_bfloat16* slices = nullptr;   // operand slices
    size_t slice_elems = 0;
    float* part = nullptr;             // float64 split-K partials (counted in floats)
    size_t part_elems = 0;
    int* expo = nullptr;               // per-row binary exponents
    size_t expo_elems = 0;
    int* err = nullptr;                // bounded-wait expiry flag
};
// Workspace one product takes in one piece (part: room for its largest
// split-K count).
void gemm_f64_tc_sizes(int M, int N, int K, int batch, bool reduce, size_t* slice_elems,
                       size_t* part_elems, size_t* expo_elems);
cudaError_t gemm_f64_tc(const Gemm<double>& g, const F64TcWorkspace& ws, cudaStream_t s);
// Randomised check of gemm_f64_tc against the float64 CUDA-core product.
cudaError_t gemm_f64_tc_selftest(int cases, unsigned long long seed, double* max_rel,
                                 int* failures, cudaStream_t st);

}  // namespace thc
