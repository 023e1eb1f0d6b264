// Throughput probes behind the C ABI (diagnostics; no counterpart in the
// paper): the CUDA-core FMA rates that serve as roofline denominators of the
// triangle kernels, and timed tensor-core products at a given shape.
#include <string>

#include "common.cuh"
#include "gemm_tc.cuh"

namespace thc {

void set_thread_error(const std::string& msg);

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread

template <typename T>
__global__ void k_fma_chains(T a, T b, int iters, T* out) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed pairs: fma.rn.f32x2 on kChains 64-bit registers.
__global__ void k_fma_chains_x2(float a, float b, int iters, float* out) {
    unsigned long long x[kChains], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v = (float)(threadIdx.x + c) * 1e-3f;
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
    }
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fill(float* p, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        p[i] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

__global__ void k_widen(const float* in, double* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i] * (1.0 + 1e-9 * (double)(i % 7));
}

}  // namespace
}  // namespace thc

using namespace thc;

extern "C" thc_status thc_probe_alu(int kind, double* tflops, void* stream) {
    if (kind < 0 || kind > 2 || !tflops) {
        set_thread_error("thc_probe_alu: kind must be 0, 1 or 2 and tflops non-NULL");
        return THC_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = device_sms() * 8, threads = 256;
    const int iters = kind == 0 ? 2048 : 65536;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // warm-up, then timed
        cudaEventRecord(e0, st);
        if (kind == 0)
            k_fma_chains<double><<<blocks, threads, 0, st>>>(0.999999, 1e-7, iters, (double*)out);
        else if (kind == 1)
            k_fma_chains<float><<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, iters, (float*)out);
        else
            k_fma_chains_x2<<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, iters / 2, (float*)out);
        count_launches(1);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        set_thread_error(std::string("thc_probe_alu: ") + cudaGetErrorString(e));
        return THC_ERR_CUDA;
    }
    // 2 flops per FMA lane; the packed kernel runs half the iterations on two lanes
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return THC_OK;
}

extern "C" thc_status thc_probe_gemm(int mode, int M, int N, int K, int iters, double* ms_out,
                                     void* stream) {
    if (mode < 0 || mode > 3 || M <= 0 || N <= 0 || K <= 0 || iters <= 0 || !ms_out) {
        set_thread_error("thc_probe_gemm: mode 0-3, positive sizes and iterations");
        return THC_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long nA = (long long)M * K, nB = (long long)K * N, nC = (long long)M * N;
    float *A = nullptr, *B = nullptr, *C = nullptr, *part = nullptr;
    __nv_bfloat16* pack = nullptr;
    double *Ad = nullptr, *Bd = nullptr, *Cd = nullptr;
    __nv_bfloat16* sl = nullptr;
    float* fpart = nullptr;
    int* expo = nullptr;
    int* err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PackCache cache;
    float ms = 0;
    cudaError_t e = cudaMalloc(&A, nA * 4);
    if (e == cudaSuccess) e = cudaMalloc(&B, nB * 4);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fill<<<1024, 256, 0, st>>>(A, nA, 1);
        k_fill<<<1024, 256, 0, st>>>(B, nB, 2);
        count_launches(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mode <= 2) {
        // float32 operands, bf16 hi/lo products; modes 0 and 2 keep the packed
        // operands cached (product alone), mode 1 packs them on every call.
        const int nprod = mode == 2 ? 1 : 3;
        const size_t pe = gemm_tc_pack_elems(M, N, K, 1, false);
        e = cudaMalloc(&C, nC * 4);
        if (e == cudaSuccess) e = cudaMalloc(&pack, pe * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)4 * nC * 4);
        TcWorkspace ws;
        ws.buf = pack;
        ws.elems = pe;
        ws.partial = part;
        ws.partial_elems = (size_t)4 * nC;
        ws.err = err;
        Gemm<float> g;
        g.M = M; g.N = N; g.K = K;
        g.A = View<float>{A, K, 1};
        g.B = View<float>{B, N, 1};
        g.C = C; g.ldc = N;
        PackCache* pc = nullptr;
        if (mode != 1) {
            cache.add_constant(A, (size_t)nA);
            cache.add_constant(B, (size_t)nB);
            cache.budget = (size_t)4 * (nA + nB) * 2 + (1 << 20);
            pc = &cache;
        }
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = gemm_tc(g, ws, nprod, st, pc);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) e = gemm_tc(g, ws, nprod, st, pc);
    } else if (e == cudaSuccess) {
        // float64 operands by exact integer slices
        e = cudaMalloc(&Ad, nA * 8);
        if (e == cudaSuccess) e = cudaMalloc(&Bd, nB * 8);
        if (e == cudaSuccess) e = cudaMalloc(&Cd, nC * 8);
        size_t se = 0, pe = 0, ee = 0;
        gemm_f64_tc_sizes(M, N, K, 1, false, &se, &pe, &ee);
        if (e == cudaSuccess) e = cudaMalloc(&sl, se * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMalloc(&fpart, pe * 4);
        if (e == cudaSuccess) e = cudaMalloc(&expo, ee * sizeof(int));
        if (e == cudaSuccess) {
            k_widen<<<1024, 256, 0, st>>>(A, Ad, nA);
            k_widen<<<1024, 256, 0, st>>>(B, Bd, nB);
            count_launches(2);
            e = cudaGetLastError();
        }
        F64TcWorkspace ws;
        ws.slices = sl; ws.slice_elems = se;
        ws.part = fpart; ws.part_elems = pe;
        ws.expo = expo; ws.expo_elems = ee;
        ws.err = err;
        Gemm<double> g;
        g.M = M; g.N = N; g.K = K;
        g.A = View<double>{Ad, K, 1};
        g.B = View<double>{Bd, N, 1};
        g.C = Cd; g.ldc = N;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = gemm_f64_tc(g, ws, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) e = gemm_f64_tc(g, ws, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cache.release();
    for (void* p : {(void*)A, (void*)B, (void*)C, (void*)part, (void*)pack, (void*)Ad, (void*)Bd,
                    (void*)Cd, (void*)sl, (void*)fpart, (void*)expo, (void*)err})
        if (p) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_thread_error(std::string("thc_probe_gemm: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
    }
    if (h) {
        set_thread_error("thc_probe_gemm: a tensor-core kernel's bounded wait expired");
        return THC_ERR_TIMEOUT;
    }
    *ms_out = ms / iters;
    return THC_OK;
}
