// Strided, batched and batch-reducing matrix product on the CUDA cores.
//
// This runs the float64 products of the CUDA-core policy, the products too
// small for the tensor-core paths, and the float32 reference path.  Every
// operand is a strided
// view, so transposes, shared (stride-0) batch operands and column slices of
// row-major arrays need no copies.  Tiles of 64 or 80 per side (chosen per
// product to pad least) x 16, 256 threads, double-buffered shared memory.
#include <algorithm>
#include <type_traits>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace thc {

namespace {
std::atomic<long long> g_launches{0};
}
long long launches() { return g_launches.load(); }
void count_launches(int n) { g_launches += n; }

namespace {
std::mutex g_optin_mu;
std::map<std::pair<int, const void*>, int> g_optin;   // (device, kernel) -> bytes
std::map<int, int> g_sms;                              // device -> SM count
}  // namespace

cudaError_t smem_optin(const void* kernel, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_optin_mu);
    auto it = g_optin.find({dev, kernel});
    if (it != g_optin.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) g_optin[{dev, kernel}] = bytes;
    return e;
}

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    std::lock_guard<std::mutex> lock(g_optin_mu);
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 152;
    g_sms[dev] = n;
    return n;
}

namespace {

constexpr int BK = 16, NT = 256;

template <typename T, int BM, int BN>
struct Smem {
    T a[2][BK][BM + 1];
    T b[2][BK][BN + 1];
};

// Element e of a BM x BK (or BN x BK) tile for thread t: e = t + 256 j,
// coalesced along whichever index of the operand is contiguous.
template <typename T, int BM, int BN>
__device__ __forceinline__ void load_tiles(const Gemm<T>& g, int b, int k0, int m0, int n0,
                                           T (&ra)[BM / 16], T (&rb)[BN / 16], bool a_kfast,
                                           bool b_kfast) {
    const int t = threadIdx.x;
    const T* A = g.A.p + (long long)b * g.sAb;
    const T* B = g.B.p + (long long)b * g.sBb;
#pragma unroll
    for (int j = 0; j < BM / 16; ++j) {
        const int e = t + NT * j;
        const int m = a_kfast ? e / BK : e % BM, k = a_kfast ? e % BK : e / BM;
        const int gm = m0 + m, gk = k0 + k;
        ra[j] = (gm < g.M && gk < g.K) ? A[gm * g.A.rs + gk * g.A.cs] : T(0);
    }
#pragma unroll
    for (int j = 0; j < BN / 16; ++j) {
        const int e = t + NT * j;
        const int n = b_kfast ? e / BK : e % BN, k = b_kfast ? e % BK : e / BN;
        const int gn = n0 + n, gk = k0 + k;
        rb[j] = (gn < g.N && gk < g.K) ? B[gk * g.B.rs + gn * g.B.cs] : T(0);
    }
}

template <typename T, int BM, int BN>
__device__ __forceinline__ void store_tiles(Smem<T, BM, BN>& sm, int buf, const T (&ra)[BM / 16],
                                            const T (&rb)[BN / 16], bool a_kfast, bool b_kfast) {
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < BM / 16; ++j) {
        const int e = t + NT * j;
        const int m = a_kfast ? e / BK : e % BM, k = a_kfast ? e % BK : e / BM;
        sm.a[buf][k][m] = ra[j];
    }
#pragma unroll
    for (int j = 0; j < BN / 16; ++j) {
        const int e = t + NT * j;
        const int n = b_kfast ? e / BK : e % BN, k = b_kfast ? e % BK : e / BN;
        sm.b[buf][k][n] = rb[j];
    }
}

// BM x BN x 16 tiles (BM, BN in {64, 80}), 256 threads, a (BM/16) x (BN/16)
// register tile per thread, double-buffered shared memory.
template <typename T, int BM, int BN>
__global__ void __launch_bounds__(NT) gemm_kernel(const Gemm<T> g) {
    __shared__ Smem<T, BM, BN> sm;
    constexpr int RI = BM / 16, RJ = BN / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool a_kfast = (g.A.cs == 1) || (g.A.rs != 1 && g.A.cs < g.A.rs);
    const bool b_kfast = (g.B.rs == 1) || (g.B.cs != 1 && g.B.rs < g.B.cs);
    T acc[RI][RJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) acc[i][j] = T(0);

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
    T ra[RI], rb[RJ];
    if (s_lo < s_hi) {
        load_tiles<T, BM, BN>(g, b_lo + s_lo / ktiles, (s_lo % ktiles) * BK, m0, n0, ra, rb,
                              a_kfast, b_kfast);
        store_tiles<T, BM, BN>(sm, 0, ra, rb, a_kfast, b_kfast);
    }
    __syncthreads();
    for (int step = s_lo; step < s_hi; ++step) {
        const int buf = (step - s_lo) & 1;
        const bool more = step + 1 < s_hi;
        if (more) {
            int nb = b_lo + (step + 1) / ktiles, nk = ((step + 1) % ktiles) * BK;
            load_tiles<T, BM, BN>(g, nb, nk, m0, n0, ra, rb, a_kfast, b_kfast);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[RI], b[RJ];
#pragma unroll
            for (int i = 0; i < RI; ++i) a[i] = sm.a[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < RJ; ++j) b[j] = sm.b[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
                for (int j = 0; j < RJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) store_tiles<T, BM, BN>(sm, buf ^ 1, ra, rb, a_kfast, b_kfast);
        __syncthreads();
    }
    if (g.splits > 1) {
        // Raw partial sums; gemm_splitk_reduce applies alpha and beta.
        T* Wp = g.ws + (long long)blockIdx.z * g.M * g.N;
#pragma unroll
        for (int i = 0; i < RI; ++i) {
            int m = m0 + ty + 16 * i;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                int n = n0 + tx + 16 * j;
                if (n < g.N) Wp[(long long)m * g.N + n] = acc[i][j];
            }
        }
        return;
    }
    T* C = g.C + (g.reduce ? 0 : (long long)bz * g.sCb);
    const T alpha = T(g.alpha), beta = T(g.beta);
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
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

// C(0, n) = alpha sum_k A(0, k) B(k, n) + beta C(0, n): a row vector times a
// matrix, one thread per output column (a 64 x 64 tile would compute 64 rows
// for the one that exists).
template <typename T>
__global__ void k_gemv_row(Gemm<T> g) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.N;
         n += (long long)gridDim.x * blockDim.x) {
        T acc = 0;
        for (int k = 0; k < g.K; ++k)
            acc += g.A.p[(long long)k * g.A.cs] * g.B.p[(long long)k * g.B.rs + n * g.B.cs];
        T* c = g.C + n;
        *c = g.beta != 0.0 ? (T)(g.alpha * acc + g.beta * *c) : (T)(g.alpha * acc);
    }
}

// C(m, 0) = alpha sum_k A(m, k) B(k, 0) + beta C(m, 0): a matrix times a
// vector, one 256-thread block per output row (the rows are few and long
// here), fixed-order reduction.
template <typename T>
__global__ void k_gemv_col(Gemm<T> g) {
    __shared__ T part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long m = blockIdx.x; m < g.M; m += gridDim.x) {
        T acc = 0;
        for (int k = threadIdx.x; k < g.K; k += blockDim.x)
            acc += g.A.p[m * g.A.rs + (long long)k * g.A.cs] * g.B.p[(long long)k * g.B.rs];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) part[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            T sum = 0;
            for (int w = 0; w < 8; ++w) sum += part[w];
            T* c = g.C + m * g.ldc;
            *c = g.beta != 0.0 ? (T)(g.alpha * sum + g.beta * *c) : (T)(g.alpha * sum);
        }
        __syncthreads();
    }
}

// Tile edges (64 or 80 per side): the pair that pads the product least
// (e.g. 400 = 5 x 80 instead of 7 x 64 = 448), among those that still give
// two waves of blocks, directly or through split-K (ksteps 16-deep steps
// allow up to ksteps / 16 splits); 64 x 64 when none does or on a tie.
void tile_edges(long long M, long long N, long long nb, long long ksteps, int* BM, int* BN) {
    *BM = 64;
    *BN = 64;
    long long best = (long long)cdiv(M, 64) * 64 * cdiv(N, 64) * 64;
    for (int bm : {64, 80})
        for (int bn : {64, 80}) {
            const long long tiles = (long long)cdiv(M, bm) * cdiv(N, bn) * nb;
            const long long area = (long long)cdiv(M, bm) * bm * cdiv(N, bn) * bn;
            const long long reach = tiles * std::max(1LL, ksteps >= 32 ? ksteps / 16 : 1);
            if (reach >= 2 * 152 && area < best) {
                best = area;
                *BM = bm;
                *BN = bn;
            }
        }
}

template <typename T, int BM, int BN>
cudaError_t run(const Gemm<T>& g, dim3 grid, cudaStream_t s) {
    gemm_kernel<T, BM, BN><<<grid, NT, 0, s>>>(g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch(Gemm<T> g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    if (g.K <= 0) {
        g.K = 0;   // C = beta C
    }
    if (std::is_same<T, double>::value && g.batch == 1 && !g.reduce && g.K > 0 &&
        (g.M == 1 || g.N == 1)) {
        // float64 vector products (float32 tiles are cheap enough)
        if (g.M == 1) {
            k_gemv_row<T><<<(unsigned)std::min<long long>((g.N + 255) / 256, 152 * 8), 256, 0, s>>>(g);
        } else {
            k_gemv_col<T><<<(unsigned)std::min<long long>(g.M, 152 * 8), 256, 0, s>>>(g);
        }
        count_launches(1);
        return cudaGetLastError();
    }
    int BM = 64, BN = 64;
    tile_edges(g.M, g.N, g.reduce ? 1 : g.batch,
               (long long)(g.reduce ? g.batch : 1) * ((g.K + BK - 1) / BK), &BM, &BN);
    const long long tiles = (long long)cdiv(g.N, BN) * cdiv(g.M, BM) * (g.reduce ? 1 : g.batch);
    const long long ksteps = (long long)(g.reduce ? g.batch : 1) * ((g.K + BK - 1) / BK);
    int splits = 1;
    if (g.ws && tiles < kTargetBlocks && ksteps >= 8) {
        // split K (chunks of at least 4 steps) when the tiles alone leave
        // most SMs idle: a float64 tile runs at 4 G multiply-adds/s per SM
        long long want = (kTargetBlocks + tiles - 1) / tiles;
        long long cap_k = ksteps / 4;
        long long per = (long long)g.M * g.N * (g.reduce ? 1 : g.batch);
        long long cap_ws = (long long)(g.ws_elems / (size_t)per);
        splits = (int)std::max(1LL, std::min({want, cap_k, cap_ws, 64LL}));
    }
    g.splits = splits;
    dim3 grid(cdiv(g.N, BN), cdiv(g.M, BM), (g.reduce ? 1 : g.batch) * splits);
    if (grid.z > 65535 || grid.y > 65535) return cudaErrorInvalidValue;
    cudaError_t e;
    if (BM == 64 && BN == 64) e = run<T, 64, 64>(g, grid, s);
    else if (BM == 64) e = run<T, 64, 80>(g, grid, s);
    else if (BN == 64) e = run<T, 80, 64>(g, grid, s);
    else e = run<T, 80, 80>(g, grid, s);
    if (e != cudaSuccess) return e;
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
