// Float32 triangle kernel of the mixed-precision path (Alg. 6 line 11, Eq. 34):
//   H^XYZ += sum_I (E_I^XY F_I^XZ + E_I^XZ F_I^XY) G_I^YZ.
//
// t^XYZ = E^XY F^XZ + E^XZ F^XY is symmetric in (Y, Z), so a block takes a
// pair of mirror (Y, Z) tiles and one t feeds both H^XYZ (with G^YZ) and
// H^XZY (with G^ZY).  Two amplitude indices X = 2q, 2q + 1 run in the two
// lanes of packed f32x2 instructions: E and F are stored with the rows of a
// pair interleaved, E2_I[q][Y] = {E_I^{2q,Y}, E_I^{2q+1,Y}}, so that one
// 8-byte value holds both lanes.  Per (X pair, Y, Z) pair of mirror outputs
// the kernel issues one packed multiply and three packed FMAs: 2 FMA-pipe
// lanes per (I, X, Y, Z) term, where the unpaired form takes 3.
//
// Block: 16 X (8 pairs) x a mirror pair of 32 x 32 (Y, Z) tiles, 256
// threads.  Warp w takes pairs 4 (w / 4) .. + 3, Y half (w / 2) % 2 and Z
// half w % 2; lane (lx, ly, lz) = (lane / 16, lane / 4 % 4, lane % 4) owns
// the pairs 4 (w / 4) + lx + 2p (p < 2), Y = 16 ((w / 2) % 2) + 4 ly + (0..3)
// and Z = 16 (w % 2) + 4 lz + (0..3): 64 packed accumulators per thread.
// One thread streams the operands with 3-D TMA boxes (128-byte swizzle)
// through a ring of QS stages of QI grid points; every wait is bounded.
// The last warp to finish with a stage issues its refill.  Measured at
// P = 400, 400 rows X, 1200 grid points: two stages of six grid points
// 8.54 ms (0.56 of the FP32 peak in algorithmic flops), three of four 9.33,
// four of three 9.89, five of two 10.57; with the refills issued by one
// thread of warp 0 instead, 9.16, 9.85, 10.6 and 12.2 ms.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "kernels.cuh"

namespace thc {
namespace {

typedef unsigned long long f2;   // two float32 lanes: low word = lane 0 (X = 2q)

#ifndef THC_PAIR_QI
#define THC_PAIR_QI 6
#endif
#ifndef THC_PAIR_QS
#define THC_PAIR_QS 2
#endif
constexpr int QT = 32;            // Y and Z tile
constexpr int QP = 8;             // X pairs per block
constexpr int QI = THC_PAIR_QI;   // grid points per stage
constexpr int QS = THC_PAIR_QS;   // ring stages
constexpr long long kQWait = 4000000000LL;

struct QSmem {
    // E2, F2 half tiles: [stage][half][grid point][pair][16 pairs of floats]
    // (128-byte rows, 1 KB per (half, grid point)).
    f2 ey[QS][2][QI][QP][16];
    f2 ez[QS][2][QI][QP][16];
    f2 fy[QS][2][QI][QP][16];
    f2 fz[QS][2][QI][QP][16];
    float g1[QS][QI][QT][QT];   // G^YZ, rows Y
    float g2[QS][QI][QT][QT];   // G^ZY, rows Z
    unsigned long long full[QS];
    unsigned cnt[QS];     // warps done with the stage, over all its uses
    int last[QS];         // last step issued into the stage
    int fail;
};

__device__ __forceinline__ unsigned su32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool q_wait(unsigned long long* bar, unsigned parity) {
    const unsigned a = su32(bar);
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
        if (done) return true;
        if (clock64() - t0 > kQWait) return false;
    }
}

__device__ __forceinline__ void q_tma(void* dst, const CUtensorMap* m, unsigned long long* bar,
                                      int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(su32(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(c0), "r"(c1), "r"(c2),
        "r"(su32(bar))
        : "memory");
}

// 16 bytes at chunk `chunk` of 128-byte row `row` of a swizzled tile at
// shared address `tile` (chunk c of row r sits at c ^ (r & 7)).
__device__ __forceinline__ ulonglong2 lds_pairs(unsigned tile, int row, int chunk) {
    ulonglong2 v;
    const unsigned a = tile + (unsigned)(row * 128) + ((unsigned)(chunk ^ (row & 7)) << 4);
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];\n" : "=l"(v.x), "=l"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds_f4(unsigned tile, int row, int chunk) {
    float4 v;
    const unsigned a = tile + (unsigned)(row * 128) + ((unsigned)(chunk ^ (row & 7)) << 4);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}

__device__ __forceinline__ f2 bcast(float a) {
    f2 r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Grid: x = block of QP X pairs (fastest, so that the blocks running together
// share the G tiles of one mirror pair in L2), y = pair of mirror tiles.
__global__ void __launch_bounds__(256, 1)
    k_triangle_pair(float* H, const __grid_constant__ CUtensorMap tmE,
                    const __grid_constant__ CUtensorMap tmF,
                    const __grid_constant__ CUtensorMap tmG, int P, int nX, int nI, int* err) {
    extern __shared__ __align__(1024) unsigned char q_raw[];
    QSmem& sm = *reinterpret_cast<QSmem*>((reinterpret_cast<uintptr_t>(q_raw) + 1023) &
                                          ~uintptr_t(1023));
    const int nb = (P + QT - 1) / QT;
    int pidx = blockIdx.y, Yb = 0;
    while (pidx >= nb - Yb) {
        pidx -= nb - Yb;
        ++Yb;
    }
    const int Zb = Yb + pidx;
    const int Y0 = Yb * QT, Z0 = Zb * QT, q0 = blockIdx.x * QP;
    const bool diag = Yb == Zb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xs = warp >> 2, wy = (warp >> 1) & 1, wz = warp & 1;
    const int lx = lane >> 4, ly = (lane >> 2) & 3, lz = lane & 3;
    const int nst = (nI + QI - 1) / QI;
    const unsigned stage_bytes = 8u * QI * QP * 128u + 2u * QI * QT * QT * 4u;
    if (threadIdx.x == 0) {
        for (int s = 0; s < QS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&sm.full[s])));
            sm.cnt[s] = 0;
            sm.last[s] = -1;
        }
        sm.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int k) {
        const int s = k % QS, I0 = k * QI;
        sm.last[s] = k;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                         su32(&sm.full[s])),
                     "r"(stage_bytes));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            q_tma(&sm.ey[s][h][0][0][0], &tmE, &sm.full[s], Y0 + 16 * h, q0, I0);
            q_tma(&sm.ez[s][h][0][0][0], &tmE, &sm.full[s], Z0 + 16 * h, q0, I0);
            q_tma(&sm.fy[s][h][0][0][0], &tmF, &sm.full[s], Y0 + 16 * h, q0, I0);
            q_tma(&sm.fz[s][h][0][0][0], &tmF, &sm.full[s], Z0 + 16 * h, q0, I0);
        }
        q_tma(&sm.g1[s][0][0][0], &tmG, &sm.full[s], Z0, Y0, I0);
        q_tma(&sm.g2[s][0][0][0], &tmG, &sm.full[s], Y0, Z0, I0);
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < QS && j < nst; ++j) issue(j);

    f2 a1[2][4][4], a2[2][4][4];   // [p][yy][zz]: H^{X,Y,Z} and H^{X,Z,Y}
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a1[p][i][j] = a2[p][i][j] = 0ull;

    int k = 0;
    for (; k < nst; ++k) {
        const int s = k % QS;
        if (!q_wait(&sm.full[s], (k / QS) & 1)) atomicExch(&sm.fail, 1);
        if (*(volatile int*)&sm.fail) break;
#pragma unroll 1
        for (int ti = 0; ti < QI; ++ti) {
            if (k * QI + ti >= nI) break;
            const unsigned g1t = su32(&sm.g1[s][ti][0][0]), g2t = su32(&sm.g2[s][ti][0][0]);
            // G^YZ and G^ZY of the thread's 4 x 4 (Y, Z), both lanes alike
            f2 gb1[4][4], gb2[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 u = lds_f4(g1t, 16 * wy + 4 * ly + i, 4 * wz + lz);
                gb1[i][0] = bcast(u.x);
                gb1[i][1] = bcast(u.y);
                gb1[i][2] = bcast(u.z);
                gb1[i][3] = bcast(u.w);
                const float4 w = lds_f4(g2t, 16 * wz + 4 * lz + i, 4 * wy + ly);
                gb2[0][i] = bcast(w.x);
                gb2[1][i] = bcast(w.y);
                gb2[2][i] = bcast(w.z);
                gb2[3][i] = bcast(w.w);
            }
            const unsigned eyt = su32(&sm.ey[s][wy][ti][0][0]), ezt = su32(&sm.ez[s][wz][ti][0][0]);
            const unsigned fyt = su32(&sm.fy[s][wy][ti][0][0]), fzt = su32(&sm.fz[s][wz][ti][0][0]);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int q = 4 * xs + 2 * p + lx;
                f2 ey[4], fy[4], ez[4], fz[4];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const ulonglong2 e1 = lds_pairs(eyt, q, 2 * ly + hh);
                    const ulonglong2 f1 = lds_pairs(fyt, q, 2 * ly + hh);
                    const ulonglong2 e2 = lds_pairs(ezt, q, 2 * lz + hh);
                    const ulonglong2 f3 = lds_pairs(fzt, q, 2 * lz + hh);
                    ey[2 * hh] = e1.x;
                    ey[2 * hh + 1] = e1.y;
                    fy[2 * hh] = f1.x;
                    fy[2 * hh + 1] = f1.y;
                    ez[2 * hh] = e2.x;
                    ez[2 * hh + 1] = e2.y;
                    fz[2 * hh] = f3.x;
                    fz[2 * hh + 1] = f3.y;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // t = E^XY F^XZ + E^XZ F^XY for X = 2q, 2q + 1
                        f2 t = mul2(ey[i], fz[j]);
                        t = fma2(ez[j], fy[i], t);
                        a1[p][i][j] = fma2(t, gb1[i][j], a1[p][i][j]);
                        a2[p][i][j] = fma2(t, gb2[i][j], a2[p][i][j]);
                    }
            }
        }
        // The last warp to finish with the stage refills it at once with
        // step k + QS (its reads are ordered before the copy by the fences
        // and the atomic).
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const unsigned done = atomicAdd(&sm.cnt[s], 1u);
            if (done % 8u == 7u && k + QS < nst) {
                __threadfence_block();
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                issue(k + QS);
            }
        }
    }
    __syncthreads();
    if (*(volatile int*)&sm.fail) {
        if (threadIdx.x == 0) {
            // let the copies already issued land before the block exits
            for (int s = 0; s < QS; ++s) {
                const int j = *(volatile int*)&sm.last[s];
                if (j >= k) (void)q_wait(&sm.full[s], (j / QS) & 1);
            }
            atomicExch(err, 1);
        }
        return;
    }
    // On a diagonal pair both accumulators cover the same tile and count
    // every (Y, Z) twice.
    const float scale = diag ? 0.5f : 1.f;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int X = 2 * (q0 + 4 * xs + 2 * p + lx);
        const int Zs = Z0 + 16 * wz + 4 * lz;
        if (Zs >= P) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int Y = Y0 + 16 * wy + 4 * ly + i;
            if (Y >= P) continue;
            float v0[4], v1[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) upk(a1[p][i][j], v0[j], v1[j]);
#pragma unroll
            for (int L = 0; L < 2; ++L) {
                if (X + L >= nX) continue;
                const float* v = L ? v1 : v0;
                float4* h = reinterpret_cast<float4*>(H + ((long long)(X + L) * P + Y) * P + Zs);
                float4 c = *h;
                c.x += scale * v[0];
                c.y += scale * v[1];
                c.z += scale * v[2];
                c.w += scale * v[3];
                *h = c;
            }
        }
    }
    if (diag) __syncthreads();   // mirror targets overlap other threads' first targets
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int X = 2 * (q0 + 4 * xs + 2 * p + lx);
        const int Ys = Y0 + 16 * wy + 4 * ly;
        if (Ys >= P) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int Z = Z0 + 16 * wz + 4 * lz + j;
            if (Z >= P) continue;
            float v0[4], v1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) upk(a2[p][i][j], v0[i], v1[i]);
#pragma unroll
            for (int L = 0; L < 2; ++L) {
                if (X + L >= nX) continue;
                const float* v = L ? v1 : v0;
                float4* h = reinterpret_cast<float4*>(H + ((long long)(X + L) * P + Z) * P + Ys);
                float4 c = *h;
                c.x += scale * v[0];
                c.y += scale * v[1];
                c.z += scale * v[2];
                c.w += scale * v[3];
                *h = c;
            }
        }
    }
}

// In place, per slab b and row pair q: rows 2q and 2q + 1 of P floats at
// A + b stride + (2q + r) P become the pairs {A^{2q,Y}, A^{2q+1,Y}} at
// A + b stride + 2qP + 2Y.  For odd nX the last pair takes 0 in its second
// lane (its second row is the slab's padding, never read).
__global__ void __launch_bounds__(256) k_pair_rows(float* A, long long nslab, long long stride,
                                                   int nX, int P) {
    extern __shared__ float seg[];   // 2P floats
    const int nq = (nX + 1) / 2;
    for (long long w = blockIdx.x; w < nslab * nq; w += gridDim.x) {
        const long long b = w / nq;
        const int q = (int)(w % nq);
        float* base = A + b * stride + 2LL * q * P;
        const int n = 2 * q + 1 < nX ? 2 * P : P;
        for (int i = threadIdx.x; i < 2 * P; i += blockDim.x) seg[i] = i < n ? base[i] : 0.f;
        __syncthreads();
        float2* out = reinterpret_cast<float2*>(base);
        for (int y = threadIdx.x; y < P; y += blockDim.x) out[y] = make_float2(seg[y], seg[P + y]);
        __syncthreads();
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_q_encode = nullptr;
std::once_flag g_q_once;

// 3-D map (x, rows, nI) of elements of `esize` bytes (x contiguous, rows of
// x elements), box (bx, by, QI), 128-byte swizzle, zero fill outside.
cudaError_t q_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esize, long long x,
                  long long rows, int nI, int bx, int by) {
    std::call_once(g_q_once, [] {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_q_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_q_encode) return cudaErrorNotSupported;
    cuuint64_t dims[3] = {(cuuint64_t)x, (cuuint64_t)rows, (cuuint64_t)nI};
    cuuint64_t strides[2] = {(cuuint64_t)(x * esize), (cuuint64_t)(x * rows * esize)};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)QI};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_q_encode(m, dt, 3, const_cast<void*>(base), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool triangle_pair_ok(int P) { return P > 0 && P % 4 == 0 && P <= kPairMaxP; }

cudaError_t pair_rows(float* A, long long nslab, long long stride, int nX, int P,
                      cudaStream_t s) {
    if (nslab <= 0 || nX <= 0) return cudaSuccess;
    if (!triangle_pair_ok(P) || stride < (long long)(nX + (nX & 1)) * P || stride % 2)
        return cudaErrorInvalidValue;
    const long long work = nslab * ((nX + 1) / 2);
    const unsigned grid = (unsigned)std::min<long long>(work, 152LL * 8);
    const int smem = 2 * P * (int)sizeof(float);
    if (smem > 48 * 1024) {
        const cudaError_t e = smem_optin((const void*)k_pair_rows, smem);
        if (e != cudaSuccess) return e;
    }
    k_pair_rows<<<grid, 256, smem, s>>>(A, nslab, stride, nX, P);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t triangle_pair(float* H, const float2* E2, const float2* F2, const float* G, int P,
                          int nX, int nI, cudaStream_t s, int* err) {
    if (nX <= 0 || nI <= 0) return cudaSuccess;
    if (!triangle_pair_ok(P) || !err || (uintptr_t)E2 % 16 || (uintptr_t)F2 % 16 ||
        (uintptr_t)G % 16)
        return cudaErrorInvalidValue;
    const int nXp = (nX + 1) / 2;
    CUtensorMap mE, mF, mG;
    cudaError_t e = q_map(&mE, E2, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, P, nXp, nI, 16, QP);
    if (e == cudaSuccess) e = q_map(&mF, F2, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, P, nXp, nI, 16, QP);
    if (e == cudaSuccess) e = q_map(&mG, G, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P, P, nI, QT, QT);
    if (e != cudaSuccess) return e;
    const int smem = (int)sizeof(QSmem) + 1024;
    e = smem_optin((const void*)k_triangle_pair, smem);
    if (e != cudaSuccess) return e;
    const unsigned nb = cdiv(P, QT);
    dim3 grid(cdiv(nXp, QP), nb * (nb + 1) / 2);
    k_triangle_pair<<<grid, 256, smem, s>>>(H, mE, mF, mG, P, nX, nI, err);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace thc
