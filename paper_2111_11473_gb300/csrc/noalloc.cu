// thc_energy_noalloc: the closed-shell CCSD energy of a THC core without any
// device allocation, for callers that may not allocate device memory.
//
// Its scratch lives in one file-scope __device__ array (THC_NOALLOC_SCRATCH
// doubles, 16 MiB) that every GPU which loads this library holds until the
// process exits.  Host code only ever sees the array's host-side shadow, so
// the device address is fetched with cudaGetSymbolAddress once per device
// (on that device's first call, with it current) and passed to the kernels.
#include <mutex>
#include <string>

#include "common.cuh"
#include "kernels.cuh"

namespace thc {

void set_thread_error(const std::string& msg);

namespace {

__device__ __align__(256) double g_noalloc_scratch[THC_NOALLOC_SCRATCH];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__device__ double nb_block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// a^X = sum_i y_i^X M3[i][X] for one Cholesky vector (M3 = L_A y_v, o x P).
__global__ void k_energy_avec(const double* yo, const double* M3, int o, int P, double* a) {
    for (int X = blockIdx.x * blockDim.x + threadIdx.x; X < P; X += gridDim.x * blockDim.x) {
        double s = 0;
        for (int i = 0; i < o; ++i) s += yo[(long long)i * P + X] * M3[(long long)i * P + X];
        a[X] = s;
    }
}

// Partial sums of one Cholesky vector A's part of the energy,
//   part = 2 a^T Zc a - sum_XY Zc^XY B^XY B^YX + 2 (L_A . t1)^2 - sum_ij M_ij M_ji,
// with B = M3^T y_o and M = L_A t1^T (o x o).  Each of the kNoallocBlocks
// blocks takes a strided share of the P^2 (and o v, o^2) elements and writes
// one partial; the two singles pieces are formed by block 0 alone, since the
// square of L_A . t1 needs the whole dot product.
constexpr int kNoallocBlocks = 32;

__global__ void k_energy_vector(const double* B, const double* Mo, const double* LA,
                                const double* t1, const double* Zc, const double* a, int o,
                                int v, int P, double* part) {
    const long long PP = (long long)P * P;
    double acc = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < PP;
         e += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(e / P), Y = (int)(e % P);
        acc += Zc[e] * (2.0 * a[X] * a[Y] - B[e] * B[(long long)Y * P + X]);
    }
    acc = nb_block_sum(acc);
    if (blockIdx.x == 0) {
        double s1 = 0, q = 0;
        for (int e = threadIdx.x; e < o * v; e += blockDim.x) s1 += LA[e] * t1[e];
        for (int e = threadIdx.x; e < o * o; e += blockDim.x) {
            const int i = e / o, j = e % o;
            q += Mo[e] * Mo[j * o + i];
        }
        __syncthreads();
        s1 = nb_block_sum(s1);
        __syncthreads();
        q = nb_block_sum(q);
        acc += 2.0 * s1 * s1 - q;
    }
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_vector(const double* part, int n, double* out) {
    double acc = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    acc = nb_block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace
}  // namespace thc

extern "C" thc_status thc_energy_noalloc(int n_occ, int n_vir, int n_p, int n_k,
                                         const double* Y, const double* Lov,
                                         const double* Zc, const double* t1,
                                         double* energy, void* stream) {
    using namespace thc;
    const int o = n_occ, v = n_vir, P = n_p, K = n_k;
    if (o <= 0 || v <= 0 || P <= 0 || K <= 0 || !Y || !Lov || !Zc || !t1 || !energy) {
        set_thread_error("thc_energy_noalloc: non-positive size or NULL pointer");
        return THC_ERR_ARG;
    }
    // The kernels read the inputs in place: they must be device memory.
    // They must also live on the current device, whose copy of the scratch
    // array the kernels are given.
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        set_thread_error("thc_energy_noalloc: no current CUDA device");
        return THC_ERR_CUDA;
    }
    for (const double* p : {Y, Lov, Zc, t1}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            set_thread_error("thc_energy_noalloc: Y, Lov, Zc and t1 must be device memory");
            return THC_ERR_ARG;
        }
        if (a.device != cur) {
            set_thread_error("thc_energy_noalloc: Y, Lov, Zc and t1 must be memory of the "
                             "current device (" + std::to_string(cur) + "), not of device " +
                             std::to_string(a.device));
            return THC_ERR_ARG;
        }
    }
    // Scratch layout: M3 (o P) | B (P P) | a (P) | Mo (o o) | part (32 K) | result (1)
    const long long need = (long long)o * P + (long long)P * P + P + (long long)o * o +
                           (long long)kNoallocBlocks * K + 1;
    if (need > (long long)THC_NOALLOC_SCRATCH) {
        set_thread_error("thc_energy_noalloc: o*P + P*P + P + o*o + 32*K + 1 = " +
                         std::to_string(need) + " doubles exceeds the fixed scratch of " +
                         std::to_string((long long)THC_NOALLOC_SCRATCH) + " doubles");
        return THC_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_thread_error(std::string("thc_energy_noalloc: cudaGetSymbolAddress: ") +
                         cudaGetErrorString(e));
        return THC_ERR_CUDA;
    }
    double* M3 = base;
    double* B = M3 + (long long)o * P;
    double* a = B + (long long)P * P;
    double* Mo = a + P;
    double* part = Mo + (long long)o * o;
    double* result = part + (long long)kNoallocBlocks * K;
    const double* yo = Y;
    const double* yv = Y + (long long)o * P;
    const long long ov = (long long)o * v;
    // Every region is overwritten before it is read; the partial sums are
    // cleared anyway so that a failed launch cannot leave stale values.
    e = cudaMemsetAsync(part, 0, sizeof(double) * ((long long)kNoallocBlocks * K + 1), st);
    for (int A = 0; A < K && e == cudaSuccess; ++A) {
        const double* LA = Lov + A * ov;
        Gemm<double> g;   // M3 = L_A y_v
        g.M = o; g.N = P; g.K = v; g.A = View<double>{LA, v, 1}; g.B = View<double>{yv, P, 1};
        g.C = M3; g.ldc = P;
        e = gemm_simt(g, st);
        if (e != cudaSuccess) break;
        Gemm<double> h;   // B = M3^T y_o
        h.M = P; h.N = P; h.K = o; h.A = View<double>{M3, 1, P}; h.B = View<double>{yo, P, 1};
        h.C = B; h.ldc = P;
        e = gemm_simt(h, st);
        if (e != cudaSuccess) break;
        Gemm<double> m;   // Mo = L_A t1^T
        m.M = o; m.N = o; m.K = v; m.A = View<double>{LA, v, 1}; m.B = View<double>{t1, 1, v};
        m.C = Mo; m.ldc = o;
        e = gemm_simt(m, st);
        if (e != cudaSuccess) break;
        k_energy_avec<<<(P + 255) / 256, 256, 0, st>>>(yo, M3, o, P, a);
        k_energy_vector<<<kNoallocBlocks, 256, 0, st>>>(B, Mo, LA, t1, Zc, a, o, v, P,
                                                        part + (long long)kNoallocBlocks * A);
        count_launches(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_sum_vector<<<1, 256, 0, st>>>(part, kNoallocBlocks * K, result);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(energy, result, sizeof(double), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_thread_error(std::string("thc_energy_noalloc: ") + cudaGetErrorString(e));
        return THC_ERR_CUDA;
    }
    return THC_OK;
}
