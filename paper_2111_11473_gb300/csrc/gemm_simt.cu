// Strided, batched and batch-reducing matrix product on the CUDA cores.
//
// This is the float64 contraction engine of the library (tcgen05 has no
// float64 kind) and the float32 reference path.  Every operand is a strided
// view, so transposes, shared (stride-0) batch operands and column slices of
// row-major arrays need no copies.  Tile 64 x 64 x 16, 256 threads, a 4 x 4
// register tile per thread, double-buffered shared memory.
#include <algorithm>

#include <atomic>

#include "common.cuh"

namespace thc {

namespace {
std::atomic<long long> g_launches{0};
}
long long launches() { return g_launches.load(); }
void count_launches(int n) { g_launches += n; }

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
struct Smem {
    T a[2][BK][BM + 1];
    T b[2][BK][BN + 1];
};

template <typename T>
__device__ __forceinline__ void load_tiles(const Gemm<T>& g, int b, int k0,
                                           int m0, int n0, T (&ra)[4],
                                           T (&rb)[4], bool a_kfast,
                                           bool b_kfast) {
    const int t = threadIdx.x;
    const T* A = g.A.p + (long long)b * g.sAb;
    const T* B = g.B.p + (long long)b * g.sBb;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int m, k;
        if (a_kfast) { k = t & 15; m = (t >> 4) + 16 * j; }
        else         { m = t & 63; k = (t >> 6) + 4 * j; }
        int gm = m0 + m, gk = k0 + k;
        ra[j] = (gm < g.M && gk < g.K) ? A[gm * g.A.rs + gk * g.A.cs] : T(0);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int n, k;
        if (b_kfast) { k = t & 15; n = (t >> 4) + 16 * j; }
        else         { n = t & 63; k = (t >> 6) + 4 * j; }
        int gn = n0 + n, gk = k0 + k;
        rb[j] = (gn < g.N && gk < g.K) ? B[gk * g.B.rs + gn * g.B.cs] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store_tiles(Smem<T>& sm, int buf, const T (&ra)[4],
                                            const T (&rb)[4], bool a_kfast,
                                            bool b_kfast) {
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int m, k;
        if (a_kfast) { k = t & 15; m = (t >> 4) + 16 * j; }
        else         { m = t & 63; k = (t >> 6) + 4 * j; }
        sm.a[buf][k][m] = ra[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int n, k;
        if (b_kfast) { k = t & 15; n = (t >> 4) + 16 * j; }
        else         { n = t & 63; k = (t >> 6) + 4 * j; }
        sm.b[buf][k][n] = rb[j];
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) gemm_kernel(const Gemm<T> g) {
    __shared__ Smem<T> sm;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool a_kfast = (g.A.cs == 1) || (g.A.rs != 1 && g.A.cs < g.A.rs);
    const bool b_kfast = (g.B.rs == 1) || (g.B.cs != 1 && g.B.rs < g.B.cs);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    // blockIdx.z = (batch index, split index); a split owns a contiguous
    // range of the (batch, k-tile) steps it accumulates.
    const int split = blockIdx.z % g.splits;
    const int bz = blockIdx.z / g.splits;
    const int b_lo = g.reduce ? 0 : bz;
    const int ktiles = (g.K + BK - 1) / BK;
    const int nsteps = (g.reduce ? g.batch : 1) * ktiles;
    const int chunk = (nsteps + g.splits - 1) / g.splits;
    const int s_lo = split * chunk;
    const int s_hi = min(nsteps, s_lo + chunk);
    T ra[4], rb[4];
    if (s_lo < s_hi) {
        load_tiles(g, b_lo + s_lo / ktiles, (s_lo % ktiles) * BK, m0, n0, ra, rb,
                   a_kfast, b_kfast);
        store_tiles(sm, 0, ra, rb, a_kfast, b_kfast);
    }
    __syncthreads();
    for (int step = s_lo; step < s_hi; ++step) {
        const int buf = (step - s_lo) & 1;
        const bool more = step + 1 < s_hi;
        if (more) {
            int nb = b_lo + (step + 1) / ktiles, nk = ((step + 1) % ktiles) * BK;
            load_tiles(g, nb, nk, m0, n0, ra, rb, a_kfast, b_kfast);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sm.a[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sm.b[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) store_tiles(sm, buf ^ 1, ra, rb, a_kfast, b_kfast);
        __syncthreads();
    }
    if (g.splits > 1) {
        // Raw partial sums; gemm_splitk_reduce applies alpha and beta.
        T* Wp = g.ws + (long long)blockIdx.z * g.M * g.N;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int m = m0 + ty + 16 * i;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int n = n0 + tx + 16 * j;
                if (n < g.N) Wp[(long long)m * g.N + n] = acc[i][j];
            }
        }
        return;
    }
    T* C = g.C + (g.reduce ? 0 : (long long)bz * g.sCb);
    const T alpha = T(g.alpha), beta = T(g.beta);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            T* c = C + (long long)m * g.ldc + n;
            T val = alpha * acc[i][j];
            if (g.beta != 0.0) val = fma(beta, *c, val);
            *c = val;
        }
    }
}

template <typename T>
__global__ void gemm_splitk_reduce(const Gemm<T> g) {
    const long long MN = (long long)g.M * g.N;
    const int nb = g.reduce ? 1 : g.batch;
    const long long total = MN * nb;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(idx / MN);
        const long long e = idx % MN;
        const int m = (int)(e / g.N), n = (int)(e % g.N);
        T acc = 0;
        for (int s = 0; s < g.splits; ++s) acc += g.ws[((long long)b * g.splits + s) * MN + e];
        T* c = g.C + (g.reduce ? 0 : (long long)b * g.sCb) + (long long)m * g.ldc + n;
        T val = T(g.alpha) * acc;
        if (g.beta != 0.0) val = fma(T(g.beta), *c, val);
        *c = val;
    }
}

constexpr int kTargetBlocks = 2 * 152;

template <typename T>
cudaError_t launch(Gemm<T> g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    if (g.K <= 0) {
        g.K = 0;   // C = beta C
    }
    const long long tiles = (long long)cdiv(g.N, BN) * cdiv(g.M, BM) * (g.reduce ? 1 : g.batch);
    const long long ksteps = (long long)(g.reduce ? g.batch : 1) * ((g.K + BK - 1) / BK);
    int splits = 1;
    if (g.ws && tiles < kTargetBlocks && ksteps >= 32) {
        long long want = (kTargetBlocks + tiles - 1) / tiles;
        long long cap_k = ksteps / 16;
        long long per = (long long)g.M * g.N * (g.reduce ? 1 : g.batch);
        long long cap_ws = (long long)(g.ws_elems / (size_t)per);
        splits = (int)std::max(1LL, std::min({want, cap_k, cap_ws, 64LL}));
    }
    g.splits = splits;
    dim3 grid(cdiv(g.N, BN), cdiv(g.M, BM), (g.reduce ? 1 : g.batch) * splits);
    if (grid.z > 65535 || grid.y > 65535) return cudaErrorInvalidValue;
    gemm_kernel<T><<<grid, NT, 0, s>>>(g);
    count_launches(splits > 1 ? 2 : 1);
    if (splits > 1) {
        long long total = (long long)g.M * g.N * (g.reduce ? 1 : g.batch);
        unsigned nbk = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 32);
        gemm_splitk_reduce<T><<<nbk, 256, 0, s>>>(g);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_simt(const Gemm<double>& g, cudaStream_t s) { return launch(g, s); }
cudaError_t gemm_simt(const Gemm<float>& g, cudaStream_t s) { return launch(g, s); }

}  // namespace thc
