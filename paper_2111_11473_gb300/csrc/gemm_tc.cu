// Tensor-core (tcgen05) matrix product for the mixed-precision path.
//
// C = alpha * A B + beta * C with float32 operands and output.  Each operand
// is split into bf16 hi/lo parts (x = hi + lo to 2^-17 relative) by a pack
// pass that also makes it K-major and pads it to the tile grid.  The product
// kernel runs hi*hi + hi*lo + lo*hi (or hi*hi only) as tcgen05.mma kind::f16
// with a float32 accumulator in tensor memory:
//   - TMA (cp.async.bulk.tensor, 128-byte swizzle) stages 128 x 64 tiles of
//     both operands through a 3-deep shared-memory ring on mbarriers;
//   - one elected thread issues the MMAs and commits each stage back to the
//     producer; a final commit releases the epilogue;
//   - four warps read the 128 x BN accumulator with tcgen05.ld and write C.
// Every mbarrier wait is bounded: on expiry the kernel raises an error flag
// that the host turns into THC_ERR_TIMEOUT, and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "gemm_tc.cuh"

namespace thc {
namespace {

constexpr int BM = 128;          // UMMA M (rows of the accumulator)
constexpr int BK = 64;           // K per stage: one 128-byte swizzle atom of bf16
constexpr int UK = 16;           // K per tcgen05.mma for 16-bit inputs
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes));
}

// Parity wait bounded by a clock64 budget; returns false if it expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: bf16 A and B, float32 D, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Shared-memory ring depth per tile width (a stage holds the 128 x 64 hi/lo
// tiles of A and the BN x 64 hi/lo tiles of B).
template <int BN>
struct TcStages {
    static constexpr int value = BN == 128 ? 3 : (BN == 64 ? 4 : 5);
};

template <int BN>
struct TcSmem {
    static constexpr int ST = TcStages<BN>::value;
    __nv_bfloat16 a_hi[ST][BM * BK];
    __nv_bfloat16 a_lo[ST][BM * BK];
    __nv_bfloat16 b_hi[ST][BN * BK];
    __nv_bfloat16 b_lo[ST][BN * BK];
    uint64_t full[ST];
    uint64_t empty[ST];
    uint64_t acc_full[2];     // accumulator buffer b holds a finished tile
    uint64_t acc_empty[2];    // the epilogue has drained accumulator buffer b
    float epi[4][32 * 33];    // per epilogue warp: a 32 x 32 tile, padded rows
    uint64_t drain;
    uint32_t tmem;
    int fail;
};

constexpr int kEpiWarps = 4;
constexpr int kTcThreads = 64 + 32 * kEpiWarps;   // producer, MMA issuer, epilogue

struct TcArgs {
    int M, N;              // real accumulator rows (UMMA M side) and columns
    int nbo;               // output batches
    int ksteps;            // 64-wide K steps per output batch
    int splits;
    int mblocks, nblocks;
    long long ntiles;      // mblocks * nblocks * nbo * splits
    float* C;              // output (or partials when splits > 1)
    long long crs, ccs, cbs;   // C(i, j) of batch b at C[b*cbs + i*crs + j*ccs]
    float alpha, beta;
    int nprod;
    int a_bcast, b_bcast;  // operand shared by every batch: packed once, batch coord 0
    int* err;
};

struct TileCoord {
    int m0, n0, bo, split, k_lo, nk;
};

__device__ __forceinline__ TileCoord tile_coord(const TcArgs& a, long long t, int BN) {
    TileCoord c;
    const int splits = a.splits, ksteps = a.ksteps;
    const int nbk = (int)(t % a.nblocks);
    long long r = t / a.nblocks;
    const int mbk = (int)(r % a.mblocks);
    r /= a.mblocks;
    c.bo = (int)(r / splits);
    c.split = (int)(r % splits);
    c.m0 = mbk * BM;
    c.n0 = nbk * BN;
    const int chunk = (ksteps + splits - 1) / splits;
    c.k_lo = c.split * chunk;
    c.nk = max(0, min(ksteps, c.k_lo + chunk) - c.k_lo);
    return c;
}

// Bounded wait that also gives up once another role has failed.
__device__ __forceinline__ bool mbar_wait_or_fail(uint64_t* bar, uint32_t parity,
                                                  volatile int* fail) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
        if (done) return true;
        if (*fail) return false;
        if (clock64() - t0 > kWaitCycles) {
            atomicExch((int*)fail, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent warp-specialised product: warp 0 streams operand tiles with TMA,
// warp 1 issues the MMAs into one of two tensor-memory accumulators, and
// warps 2-5 drain the other accumulator to C, so that the epilogue of one
// tile overlaps the main loop of the next.  Tiles are taken round-robin.
template <int BN, bool RMW>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              const TcArgs args) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    // 1024-byte alignment of the tile ring (required by the 128-byte swizzle)
    using Sm = TcSmem<BN>;
    constexpr int ST = Sm::ST;
    Sm& sm = *reinterpret_cast<Sm*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) &
                                    ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t kCols = 2 * BN < 32 ? 32 : 2 * BN;
    volatile int* fail = &sm.fail;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm.acc_full[b], 1);
            mbar_init(&sm.acc_empty[b], kEpiWarps);
        }
        mbar_init(&sm.drain, 1);
        sm.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sm.tmem;
    const uint32_t a_bytes = BM * BK * 2, b_bytes = BN * BK * 2;
    const uint32_t stage_bytes = (args.nprod == 3 ? 2 : 1) * (a_bytes + b_bytes);

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            long long it = 0;
            long long last[ST];
            for (int s = 0; s < ST; ++s) last[s] = -1;
            for (long long t = blockIdx.x; t < args.ntiles && !*fail; t += gridDim.x) {
                const TileCoord c = tile_coord(args, t, BN);
                const int ba = args.a_bcast ? 0 : c.bo, bb = args.b_bcast ? 0 : c.bo;
                for (int i = 0; i < c.nk; ++i, ++it) {
                    const int s = (int)(it % ST);
                    if (it >= ST && !mbar_wait_or_fail(&sm.empty[s], (uint32_t)(((it / ST) - 1) & 1), fail))
                        break;
                    const int kc = (c.k_lo + i) * BK;
                    mbar_expect_tx(&sm.full[s], stage_bytes);
                    tma_load_3d(sm.a_hi[s], &ta_hi, &sm.full[s], kc, c.m0, ba);
                    tma_load_3d(sm.b_hi[s], &tb_hi, &sm.full[s], kc, c.n0, bb);
                    if (args.nprod == 3) {
                        tma_load_3d(sm.a_lo[s], &ta_lo, &sm.full[s], kc, c.m0, ba);
                        tma_load_3d(sm.b_lo[s], &tb_lo, &sm.full[s], kc, c.n0, bb);
                    }
                    last[s] = it;
                }
            }
            // Every load this thread issued has landed before the CTA exits
            // (immediate unless a wait above gave up).
            for (int s = 0; s < ST; ++s)
                if (last[s] >= 0) mbar_wait(&sm.full[s], (uint32_t)((last[s] / ST) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = instr_desc(BM, BN);
            long long it = 0;
            int tl = 0;
            for (long long t = blockIdx.x; t < args.ntiles && !*fail; t += gridDim.x, ++tl) {
                const TileCoord c = tile_coord(args, t, BN);
                const int buf = tl & 1;
                if (tl >= 2 && !mbar_wait_or_fail(&sm.acc_empty[buf], (uint32_t)(((tl >> 1) - 1) & 1), fail))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t dst = tmem + (uint32_t)(buf * BN);
                bool ok = true;
                for (int i = 0; i < c.nk; ++i, ++it) {
                    const int s = (int)(it % ST);
                    if (!mbar_wait_or_fail(&sm.full[s], (uint32_t)((it / ST) & 1), fail)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t ah = smem_u32(sm.a_hi[s]), bh = smem_u32(sm.b_hi[s]);
                    const uint32_t al = smem_u32(sm.a_lo[s]), bl = smem_u32(sm.b_lo[s]);
#pragma unroll
                    for (int kk = 0; kk < BK / UK; ++kk) {
                        const uint32_t off = kk * UK * 2;   // bytes along K inside the swizzle atom
                        const uint32_t acc0 = (i > 0 || kk > 0) ? 1u : 0u;
                        mma_bf16(dst, smem_desc(ah + off), smem_desc(bh + off), idesc, acc0);
                        if (args.nprod == 3) {
                            mma_bf16(dst, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
                            mma_bf16(dst, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
                        }
                    }
                    mma_commit(&sm.empty[s]);
                }
                if (!ok) break;
                mma_commit(&sm.acc_full[buf]);
            }
            // All MMAs this thread issued have completed before TMEM is freed.
            mma_commit(&sm.drain);
            mbar_wait(&sm.drain, 0);
        }
    } else {
        // Epilogue: warp w reads accumulator lanes 32 (w % 4) .. 32 (w % 4) + 31
        // in 32-column chunks; a row-major C is written through a shared-memory
        // transpose so that every store instruction covers one 128-byte row.
        const int q = warp & 3;
        float* stg = sm.epi[q];
        int tl = 0;
        for (long long t = blockIdx.x; t < args.ntiles; t += gridDim.x, ++tl) {
            const TileCoord c = tile_coord(args, t, BN);
            const int buf = tl & 1;
            if (!mbar_wait_or_fail(&sm.acc_full[buf], (uint32_t)((tl >> 1) & 1), fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            float* Cb = args.C + (long long)c.bo * args.cbs +
                        (args.splits > 1 ? (long long)c.split * args.nbo * args.cbs : 0);
            const int i_base = c.m0 + q * 32;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32"
                    " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
                      "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
                      "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                const int j0 = c.n0 + c0;
                // RMW (beta != 0, no split): the 32 old values of C are loaded
                // before any is used, so that their latencies overlap.
                constexpr bool rmw = RMW;
                if (args.ccs == 1) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        stg[lane * 33 + j] = c.nk > 0 ? __uint_as_float(r[j]) : 0.f;
                    __syncwarp();
                    const int j = j0 + lane;
                    const bool jok = j < args.N;
                    float old[32];
                    if constexpr (rmw) {
#pragma unroll
                        for (int rr = 0; rr < 32; ++rr) {
                            const int i = i_base + rr;
                            old[rr] = (jok && i < args.M) ? Cb[(long long)i * args.crs + j] : 0.f;
                        }
                    }
                    if constexpr (rmw) {
#pragma unroll
                        for (int rr = 0; rr < 32; ++rr) {
                            const int i = i_base + rr;
                            if (i < args.M && jok)
                                Cb[(long long)i * args.crs + j] =
                                    fmaf(args.beta, old[rr], args.alpha * stg[rr * 33 + lane]);
                        }
                    } else {
#pragma unroll 4
                        for (int rr = 0; rr < 32; ++rr) {
                            const int i = i_base + rr;
                            if (i < args.M && jok) {
                                const float val = stg[rr * 33 + lane];
                                Cb[(long long)i * args.crs + j] =
                                    args.splits > 1 ? val : args.alpha * val;
                            }
                        }
                    }
                    __syncwarp();
                } else {
                    const int i = i_base + lane;
                    if (i < args.M) {
                        float old[32];
                        if constexpr (rmw) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                old[j] = (j0 + j < args.N)
                                             ? Cb[(long long)i * args.crs + (long long)(j0 + j) * args.ccs]
                                             : 0.f;
                        }
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (j0 + j < args.N) {
                                const float val = c.nk > 0 ? __uint_as_float(r[j]) : 0.f;
                                float* p = Cb + (long long)i * args.crs + (long long)(j0 + j) * args.ccs;
                                if constexpr (rmw) *p = fmaf(args.beta, old[j], args.alpha * val);
                                else *p = args.splits > 1 ? val : args.alpha * val;
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acc_empty[buf]);
        }
    }
    __syncthreads();
    if (sm.fail && threadIdx.x == 0) atomicExch(args.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kCols));
}

// Pack a strided float32 operand into bf16 hi/lo, K-major, padded:
// out[bo][r][kb*Kp + k] = split(src(b, r, k)), r < Rp, k < Kp, with
// (bo, kb) = (b, 0) for batched products and (0, b) for batch-reduced ones.
// A 32 (r) x 64 (k) tile goes through shared memory so that the global reads
// run along whichever index of the source is contiguous, and every thread
// then writes 8 consecutive k of one row as one 16-byte store of hi and lo.
constexpr int PK_R = 32, PK_K = 64;

__global__ void __launch_bounds__(256) k_pack(const float* src, long long rs, long long ks,
                                              long long bs, int R, int Kd, int nb, int Rp, int Kp,
                                              int reduce, __nv_bfloat16* hi, __nv_bfloat16* lo) {
    __shared__ float tile[PK_R][PK_K + 1];
    const int b = blockIdx.z;
    const int k0 = blockIdx.x * PK_K;
    const float* s = src + (long long)b * bs;
    const bool kfast = ks <= rs;
    const long long Ktot = reduce ? (long long)nb * Kp : Kp;
    const int bo = reduce ? 0 : b, kb = reduce ? b : 0;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int r0 = blockIdx.y * PK_R; r0 < Rp; r0 += gridDim.y * PK_R) {
        if (kfast) {
            // warp w reads rows w, w + 8, ...; lanes run along k (two halves of 32)
            for (int rr = warp; rr < PK_R; rr += 8) {
                const int r = r0 + rr;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = k0 + h * 32 + lane;
                    tile[rr][h * 32 + lane] =
                        (r < R && k < Kd) ? s[(long long)r * rs + (long long)k * ks] : 0.f;
                }
            }
        } else {
            // warp w reads columns w, w + 8, ...; lanes run along r
            for (int kk = warp; kk < PK_K; kk += 8) {
                const int r = r0 + lane, k = k0 + kk;
                tile[lane][kk] = (r < R && k < Kd) ? s[(long long)r * rs + (long long)k * ks] : 0.f;
            }
        }
        __syncthreads();
        {
            const int rr = t >> 3, oct = t & 7;   // 32 rows x 8 octets of k
            const int r = r0 + rr, k = k0 + oct * 8;
            if (r < Rp && k < Kp) {
                union { __nv_bfloat16 b[8]; uint4 u; } vh, vl;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float v = tile[rr][oct * 8 + e];
                    const __nv_bfloat16 hh = __float2bfloat16_rn(v);
                    vh.b[e] = hh;
                    vl.b[e] = __float2bfloat16_rn(v - __bfloat162float(hh));
                }
                const long long o = ((long long)bo * Rp + r) * Ktot + (long long)kb * Kp + k;
                *reinterpret_cast<uint4*>(hi + o) = vh.u;
                if (lo) *reinterpret_cast<uint4*>(lo + o) = vl.u;
            }
        }
        __syncthreads();
    }
}

__global__ void k_splitk_sum(const float* part, int splits, int nbo, int M, int N,
                             long long pcbs, float* C, long long crs, long long ccs,
                             long long cbs, float alpha, float beta) {
    const long long MN = (long long)M * N, total = MN * nbo;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(idx / MN);
        const long long e = idx % MN;
        const int i = (int)(e / N), j = (int)(e % N);
        float acc = 0.f;
        for (int s = 0; s < splits; ++s)
            acc += part[((long long)s * nbo + b) * pcbs + (long long)i * N + j];
        float* c = C + (long long)b * cbs + (long long)i * crs + (long long)j * ccs;
        *c = beta != 0.f ? fmaf(beta, *c, alpha * acc) : alpha * acc;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t get_encode() {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// 3-D map over bf16 data [nbo][rows][Ktot] with boxes of 64 (K) x box_rows.
cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, long long Ktot, long long rows,
                     int nbo, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)Ktot, (cuuint64_t)rows, (cuuint64_t)nbo};
    cuuint64_t strides[2] = {(cuuint64_t)(Ktot * 2), (cuuint64_t)(Ktot * 2 * rows)};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
cudaError_t launch_tc(const CUtensorMap* maps, const TcArgs& a, cudaStream_t s) {
    const int smem = (int)sizeof(TcSmem<BN>) + 1024;
    cudaError_t e = smem_optin((const void*)k_gemm_tc<BN, false>, smem);
    if (e == cudaSuccess) e = smem_optin((const void*)k_gemm_tc<BN, true>, smem);
    if (e != cudaSuccess) return e;
    const long long sms = device_sms();
    const unsigned grid = (unsigned)std::min<long long>(a.ntiles, sms);
    if (a.splits == 1 && a.beta != 0.f)
        k_gemm_tc<BN, true><<<grid, kTcThreads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
    else
        k_gemm_tc<BN, false><<<grid, kTcThreads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
    count_launches(1);
    return cudaGetLastError();
}

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

// Self-test of the bounded-wait path: thread 0 waits on an mbarrier that is
// completed only if `complete` is set, with a budget of `cycles`; on expiry
// it raises *flag, as every production wait does, and returns.
__global__ void k_wait_selftest(int complete, long long cycles, int* flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (complete) mbar_arrive(&bar);
    const uint32_t a = smem_u32(&bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(0u));
        if (done) return;
        if (clock64() - t0 > cycles) {
            atomicExch(flag, 1);
            return;
        }
    }
}

}  // namespace

cudaError_t wait_selftest(int complete, long long cycles, int* flag, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(complete, cycles, flag);
    count_launches(1);
    return cudaGetLastError();
}

size_t gemm_tc_pack_elems(int M, int N, int K, int batch, bool reduce) {
    // Worst case over the two orientations (both sides padded to 128).
    const long long Kp = rup(std::max(K, 1), BK);
    const long long Rm = rup(M, 128), Rn = rup(N, 128);
    return (size_t)(2 * (Rm + Rn) * Kp * batch);
}

void PackCache::release() {
    for (Entry& e : entries) cudaFree(e.hi);
    entries.clear();
    constant.clear();
    bytes = 0;
}

namespace {

// Pack one operand into the workspace, or (use_cache) take it from the cache
// of constant packs, packing it there on first use.  A cached operand that
// cannot be stored (budget or allocation) is an error, never a workspace
// write: the workspace was sized without it.
cudaError_t pack_operand(const float* p, long long rs, long long cs, long long bs, int R, int Kd,
                         int nb_eff, int nb_grid, int Rp, int Kp, int reduce, int nprod,
                         __nv_bfloat16* ws_hi, __nv_bfloat16* ws_lo, bool use_cache,
                         PackCache* cache, cudaStream_t s, __nv_bfloat16** out_hi,
                         __nv_bfloat16** out_lo) {
    const dim3 grid(cdiv(Kp, PK_K), std::min<unsigned>(cdiv(Rp, PK_R), 65535), nb_grid);
    if (use_cache) {
        for (const PackCache::Entry& e : cache->entries)
            if (e.p == p && e.rs == rs && e.cs == cs && e.bs == bs && e.R == R && e.Kd == Kd &&
                e.nb == nb_eff && e.Rp == Rp && e.Kp == Kp && e.reduce == reduce &&
                e.nprod == nprod) {
                *out_hi = e.hi;
                *out_lo = e.lo;
                return cudaSuccess;
            }
        const long long Ktot = reduce ? (long long)nb_eff * Kp : Kp;
        const size_t elems = (size_t)Rp * Ktot * (reduce ? 1 : nb_grid);
        const size_t bytes = elems * 2 * (nprod == 3 ? 2 : 1);
        if (cache->bytes + bytes > cache->budget) return cudaErrorMemoryAllocation;
        __nv_bfloat16* buf = nullptr;
        if (cudaMalloc(&buf, bytes) != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorMemoryAllocation;
        }
        PackCache::Entry e{p, rs, cs, bs, R, Kd, nb_eff, Rp, Kp, reduce, nprod, buf,
                           nprod == 3 ? buf + elems : nullptr};
        k_pack<<<grid, 256, 0, s>>>(p, rs, cs, bs, R, Kd, nb_eff, Rp, Kp, reduce, e.hi, e.lo);
        count_launches(1);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) {
            cudaFree(buf);
            return err;
        }
        cache->entries.push_back(e);
        cache->bytes += bytes;
        *out_hi = e.hi;
        *out_lo = e.lo;
        return cudaSuccess;
    }
    k_pack<<<grid, 256, 0, s>>>(p, rs, cs, bs, R, Kd, nb_eff, Rp, Kp, reduce, ws_hi, ws_lo);
    count_launches(1);
    *out_hi = ws_hi;
    *out_lo = ws_lo;
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_tc(const Gemm<float>& g, const TcWorkspace& ws, int nprod, cudaStream_t s,
                    PackCache* cache) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    // Orientation: the UMMA M side (128-row tiles) takes the larger of M, N.
    const bool swap = g.N > g.M;
    const int Mr = swap ? g.N : g.M, Nr = swap ? g.M : g.N;
    int BN = 128;
    if (Nr <= 32) BN = 32;
    else if (Nr <= 64) BN = 64;
    const long long Kp = rup(std::max(g.K, 1), BK);
    const int nb = g.batch;
    const int nbo = g.reduce ? 1 : nb;
    const long long Ktot = g.reduce ? Kp * nb : Kp;
    const long long RpA = rup(Mr, BM), RpB = rup(Nr, BN);
    // Operand views: UMMA-A rows r, K index k.
    // Unswapped: A side = A(m, k), B side = B(k, n) read as (n, k).
    View<float> va = g.A, vb{g.B.p, g.B.cs, g.B.rs};
    long long sa = g.sAb, sb = g.sBb;
    if (swap) {
        std::swap(va, vb);
        std::swap(sa, sb);
    }
    const bool a_bc = !g.reduce && nb > 1 && sa == 0;
    const bool b_bc = !g.reduce && nb > 1 && sb == 0;
    const int nba = a_bc ? 1 : nbo, nbb = b_bc ? 1 : nbo;
    const size_t needA = (size_t)(RpA * Ktot * nba), needB = (size_t)(RpB * Ktot * nbb);
    // Operands served from the cache of constant packs take no workspace.
    const int red = g.reduce ? 1 : 0;
    const size_t bytesA = needA * 2 * (nprod == 3 ? 2 : 1);
    const size_t bytesB = needB * 2 * (nprod == 3 ? 2 : 1);
    const bool a_cached = cache && cache->serves(va.p, bytesA, va.rs, va.cs, sa, Mr, g.K, nb,
                                                 (int)RpA, (int)Kp, red, nprod);
    // B is checked against the budget left after A's (possibly new) entry.
    bool b_cached = false;
    if (cache) {
        const size_t held = cache->bytes;
        if (a_cached) cache->bytes += bytesA;
        b_cached = cache->serves(vb.p, bytesB, vb.rs, vb.cs, sb, Nr, g.K, nb, (int)RpB, (int)Kp,
                                 red, nprod);
        cache->bytes = held;
    }
    const size_t need = (nprod == 3 ? 2 : 1) * ((a_cached ? 0 : needA) + (b_cached ? 0 : needB));
    if (need > ws.elems) return cudaErrorMemoryAllocation;
    // Workspace layout [A hi | B hi | A lo | B lo], cached operands omitted.
    const size_t wsA = a_cached ? 0 : needA, wsB = b_cached ? 0 : needB;
    __nv_bfloat16* a_hi = ws.buf;
    __nv_bfloat16* b_hi = a_hi + wsA;
    __nv_bfloat16* a_lo = nprod == 3 ? b_hi + wsB : nullptr;
    __nv_bfloat16* b_lo = nprod == 3 ? a_lo + wsA : nullptr;
    if ((e = pack_operand(va.p, va.rs, va.cs, sa, Mr, g.K, nb, a_bc ? 1 : nb, (int)RpA, (int)Kp,
                          red, nprod, a_hi, a_lo, a_cached, cache, s, &a_hi, &a_lo)) !=
        cudaSuccess)
        return e;
    if ((e = pack_operand(vb.p, vb.rs, vb.cs, sb, Nr, g.K, nb, b_bc ? 1 : nb, (int)RpB, (int)Kp,
                          red, nprod, b_hi, b_lo, b_cached, cache, s, &b_hi, &b_lo)) !=
        cudaSuccess)
        return e;
    CUtensorMap maps[4];
    if ((e = make_map(&maps[0], a_hi, Ktot, RpA, nba, BM)) != cudaSuccess) return e;
    if ((e = make_map(&maps[1], nprod == 3 ? a_lo : a_hi, Ktot, RpA, nba, BM)) != cudaSuccess) return e;
    if ((e = make_map(&maps[2], b_hi, Ktot, RpB, nbb, BN)) != cudaSuccess) return e;
    if ((e = make_map(&maps[3], nprod == 3 ? b_lo : b_hi, Ktot, RpB, nbb, BN)) != cudaSuccess) return e;

    TcArgs a{};
    a.M = Mr;
    a.N = Nr;
    a.nbo = nbo;
    a.ksteps = (int)(Ktot / BK);
    a.nprod = nprod;
    a.a_bcast = a_bc ? 1 : 0;
    a.b_bcast = b_bc ? 1 : 0;
    a.err = ws.err;
    a.alpha = (float)g.alpha;
    a.beta = (float)g.beta;
    // C(m, n) = g.C[b*sCb + m*ldc + n]; accumulator (i, j) is (m, n) or (n, m).
    const long long crs = swap ? 1 : g.ldc, ccs = swap ? g.ldc : 1;
    const int mblocks = (int)(RpA / BM), nblocks = (int)(RpB / BN);
    const long long tiles = (long long)mblocks * nblocks * nbo;
    int splits = 1;
    if (tiles < 152 && a.ksteps >= 8 && ws.partial) {
        splits = (int)std::min<long long>({(152 + tiles - 1) / tiles, a.ksteps / 4, 32});
        const long long per = (long long)Mr * Nr;
        while (splits > 1 && (size_t)(per * nbo * splits) > ws.partial_elems) --splits;
    }
    a.splits = splits;
    a.mblocks = mblocks;
    a.nblocks = nblocks;
    a.ntiles = tiles * splits;
    if (splits > 1) {
        a.C = ws.partial;
        a.crs = Nr;
        a.ccs = 1;
        a.cbs = (long long)Mr * Nr;
    } else {
        a.C = g.C;
        a.crs = crs;
        a.ccs = ccs;
        a.cbs = g.reduce ? 0 : g.sCb;
    }
    if (BN == 32) e = launch_tc<32>(maps, a, s);
    else if (BN == 64) e = launch_tc<64>(maps, a, s);
    else e = launch_tc<128>(maps, a, s);
    if (e != cudaSuccess) return e;
    if (splits > 1) {
        const long long total = (long long)Mr * Nr * nbo;
        const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 152 * 16);
        k_splitk_sum<<<blocks, 256, 0, s>>>(ws.partial, splits, nbo, Mr, Nr, (long long)Mr * Nr,
                                            g.C, crs, ccs, g.reduce ? 0 : g.sCb, (float)g.alpha,
                                            (float)g.beta);
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

// ---------------------------------------------------------------------------
// Float64 products on the tensor cores by exact integer slices (the splitting
// scheme of Ozaki et al.).  Every row r of an operand (UMMA orientation, K
// along the row; in a batch-reduced product the row runs over all batches) is
// scaled by 2^-e_r, e_r the binary exponent of its largest entry, so that its
// entries lie in (-1, 1), and is cut into kSlices = 8 signed 7-bit integers:
//   x = 2^e_r (sum_t a_t 2^(-7t) + r_x),   a_t in [-127, 127], |r_x| < 2^-56,
// read straight from the IEEE-754 fields (integer operations only).
// A slice is exact in bf16, a product of two is an integer below 2^14, and a
// float32 sum of at most 1024 of them is an integer below 2^24, so the tensor
// cores' float32 accumulation over K chunks of 1024 is exact.  The pairs
// (t, u) with t + u = l are one product over concatenated slices,
//   S_l = [a_1 .. a_(l-1)] [b_(l-1) .. b_1]^T   (K of (l - 1) Ktot),
// which is why A keeps its slices in order and B in reverse order along each
// row.  The levels l = 2 .. 9 (36 pairs) are combined in float64 by Horner's
// rule, sum_l 2^(-7l) S_l, and scaled by 2^(e_r + e_c).  The pairs left out
// (l >= 10) and the remainders change each product term a_rk b_kc by less
// than about 9 2^-56 = 1.2e-16 of 2^(e_r + e_c), the size of float64 rounding.
namespace {

constexpr int kSlices = 8;
constexpr int kLevels = kSlices;           // l = 2 .. kSlices + 1

// Biased exponent field of |x| (0 for zero; subnormals count as field 1).
__device__ __forceinline__ int f64_field(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    const int f = (int)(b >> 52);
    return f == 0 ? (b != 0 ? 1 : 0) : f;
}

// Load a PK_R x PK_K tile of a strided float64 operand (zeros outside) the way
// k_pack does: reads run along whichever index is contiguous.
__device__ __forceinline__ void f64_tile(double (*tile)[PK_K + 1], const double* s, long long rs,
                                         long long ks, int R, int Kd, int r0, int k0) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (ks <= rs) {
        for (int rr = warp; rr < PK_R; rr += 8) {
            const int r = r0 + rr;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k0 + h * 32 + lane;
                tile[rr][h * 32 + lane] =
                    (r < R && k < Kd) ? s[(long long)r * rs + (long long)k * ks] : 0.0;
            }
        }
    } else {
        for (int kk = warp; kk < PK_K; kk += 8) {
            const int r = r0 + lane, k = k0 + kk;
            tile[lane][kk] = (r < R && k < Kd) ? s[(long long)r * rs + (long long)k * ks] : 0.0;
        }
    }
}

// expo[bo * Rp + r] = max over the row of the biased exponent field (atomic
// over the K tiles; the array starts at zero = all-zero row).
__global__ void __launch_bounds__(256) k_row_exp(const double* src, long long rs, long long ks,
                                                 long long bs, int R, int Kd, int Rp,
                                                 int reduce, int* expo) {
    __shared__ double tile[PK_R][PK_K + 1];
    const int b = blockIdx.z;
    const int k0 = blockIdx.x * PK_K;
    const double* s = src + (long long)b * bs;
    const int bo = reduce ? 0 : b;
    const int t = threadIdx.x;
    for (int r0 = blockIdx.y * PK_R; r0 < Rp; r0 += gridDim.y * PK_R) {
        f64_tile(tile, s, rs, ks, R, Kd, r0, k0);
        __syncthreads();
        const int rr = t >> 3, oct = t & 7;
        int m = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) m = max(m, f64_field(tile[rr][oct * 8 + e]));
        // the 8 threads of a row are consecutive lanes of one warp
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o, 8));
        const int r = r0 + rr;
        if (oct == 0 && r < R && m > 0) atomicMax(&expo[(long long)bo * Rp + r], m);
        __syncthreads();
    }
}

// bf16 bits of the digit d (0 <= d <= 127) with sign bit sgn (0 or 0x8000;
// +0 for d = 0): 2^23 + d is exact in float32, the subtraction leaves d, and
// a float32 of at most 8 significant bits is its bf16 in the upper 16 bits.
__device__ __forceinline__ unsigned short digit_bf16(unsigned d, unsigned sgn) {
    const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
    return (unsigned short)((__float_as_uint(f) >> 16) | (d ? sgn : 0u));
}

// Slices of one operand: row (bo, r) holds kSlices segments of Ktot
// elements, segment q = slice q + 1 (or slice kSlices - q with reverse), in
// the packed K-major layout of k_pack (zero in the padding).  x = m 2^E with
// the 53-bit significand m; |x| 2^(56 - e) = m 2^(E - e + 56) truncated to an
// integer V < 2^56 gives the slices as its 7-bit digits.
// Five blocks of 256 threads per SM (at its natural 78 registers three fit,
// and on GB300 that measured no faster).
__global__ void __launch_bounds__(256, 5) k_slice64(const double* src, long long rs, long long ks,
                                                 long long bs, int R, int Kd, int nb, int Rp,
                                                 int Kp, int reduce, int reverse, const int* expo,
                                                 __nv_bfloat16* out) {
    __shared__ double tile[PK_R][PK_K + 1];
    const int b = blockIdx.z;
    const int k0 = blockIdx.x * PK_K;
    const double* s = src + (long long)b * bs;
    const long long Ktot = reduce ? (long long)nb * Kp : Kp;
    const int bo = reduce ? 0 : b, kb = reduce ? b : 0;
    const int t = threadIdx.x;
    for (int r0 = blockIdx.y * PK_R; r0 < Rp; r0 += gridDim.y * PK_R) {
        f64_tile(tile, s, rs, ks, R, Kd, r0, k0);
        __syncthreads();
        const int rr = t >> 3, oct = t & 7;
        const int r = r0 + rr, k = k0 + oct * 8;
        if (r < Rp && k < Kp) {
            // row exponent e = field - 1022 (|x| < 2^e); 0 = all-zero row
            const int fe = r < R ? expo[(long long)bo * Rp + r] : 0;
            union { unsigned short h[8]; uint4 u; } v[kSlices];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const unsigned long long bits =
                    (unsigned long long)__double_as_longlong(tile[rr][oct * 8 + j]);
                const int f = (int)((bits >> 52) & 0x7ff);
                const unsigned long long mant =
                    (bits & 0xfffffffffffffULL) | (f ? (1ULL << 52) : 0ULL);
                // shift = E - e + 56 with E = max(f, 1) - 1075, e = fe - 1022
                const int sh = (f ? f : 1) - fe + 3;
                unsigned long long V = 0;
                if (fe > 0 && mant != 0) {
                    if (sh >= 0) V = mant << sh;          // sh <= 3: V < 2^56
                    else if (sh > -64) V = mant >> (-sh);
                }
                const unsigned sgn = (bits >> 63) ? 0x8000u : 0u;
                // digits 0-3 in the high 28 bits of V, 4-7 in the low 28
                const unsigned vh = (unsigned)(V >> 28), vl = (unsigned)V & 0xfffffffu;
#pragma unroll
                for (int q = 0; q < kSlices; ++q) {
                    const int slice = reverse ? kSlices - 1 - q : q;      // 0-based digit
                    const unsigned dig =
                        slice < 4 ? (vh >> (7 * (3 - slice))) & 0x7fu : (vl >> (7 * (7 - slice))) & 0x7fu;
                    v[q].h[j] = digit_bf16(dig, sgn);
                }
            }
            const long long row = ((long long)bo * Rp + r) * kSlices;
#pragma unroll
            for (int q = 0; q < kSlices; ++q)
                *reinterpret_cast<uint4*>(out + (row + q) * Ktot + (long long)kb * Kp + k) =
                    v[q].u;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double pow2(int k) {
    return (k >= -1022 && k <= 1023) ? __longlong_as_double((long long)(k + 1023) << 52)
                                     : scalbn(1.0, k);
}

// 3-D map over bf16 rows of `pitch` elements of which the first kext are read.
cudaError_t make_map_pitch(CUtensorMap* map, const __nv_bfloat16* base, long long kext,
                           long long pitch, long long rows, int nbo, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)kext, (cuuint64_t)rows, (cuuint64_t)nbo};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * 2), (cuuint64_t)(pitch * 2 * rows)};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Largest split-K count of the fused product: at most 32 chunks of at least
// 8 K steps.
inline int max_f64_splits(long long Ktot) {
    return (int)std::max<long long>(1, std::min<long long>(32, Ktot / BK / 8));
}

}  // namespace

void gemm_f64_tc_sizes(int M, int N, int K, int batch, bool reduce, size_t* slice_elems,
                       size_t* part_elems, size_t* expo_elems) {
    const long long Kp = rup(std::max(K, 1), BK);
    const long long Ktot = reduce ? Kp * batch : Kp;
    const long long nbo = reduce ? 1 : batch;
    const long long Rm = rup(M, 128), Rn = rup(N, 128);
    *slice_elems = (size_t)(kSlices * (Rm + Rn) * Ktot * nbo);
    // float64 split-K partials of the fused product, counted in floats
    *part_elems = (size_t)(2LL * max_f64_splits(Ktot) * nbo * (long long)M * N);
    *expo_elems = (size_t)((Rm + Rn) * nbo);
}

// ---------------------------------------------------------------------------
// Fused float64 product: one persistent kernel per product.  For every
// 64-wide K step it loads the 8 slices of a 128-row A tile and of a 64-row B
// tile once and issues the MMAs of all 36 digit pairs (t, u), t + u <= 9,
// into eight level accumulators in tensor memory (level l = t + u at columns
// (l - 2) 64 .. (l - 2) 64 + 63: all 512 columns).  A level accumulator
// collects (l - 1) 64 products of |a_t b_u| < 2^14 per K step, so it is
// drained after c_l = floor(16 / (l - 1)) steps (at most 1024 products: an
// exact float32 integer) and restarted.  The epilogue warps combine every
// drain exactly in registers (levels 2-6 in int64, 7-9 in float32 below
// 2^-57 of the product's scale) and write the tile
// once in float64: no float32 level outputs go through memory.
// Roles: warp 0 streams slices with TMA (B slices of a K step double-
// buffered, A slices through a 4-deep ring), warp 1 issues the MMAs, warps
// 2-9 drain: warp w reads TMEM lanes 32 (w % 4) .. + 31 and columns
// 32 ((w - 2) / 4) .. + 31 of a level.  Every wait is bounded.
namespace {

constexpr int FN = 64;                    // tile columns (B rows)
#ifndef THC_F64_FA
#define THC_F64_FA 4
#endif
constexpr int FA = THC_F64_FA;            // A-slice ring depth
constexpr int kF64EpiWarps = 8;
constexpr int kF64Threads = 64 + 32 * kF64EpiWarps;

struct F64Smem {
    __nv_bfloat16 b[2][kSlices][FN * BK];   // B slices of one K step
    __nv_bfloat16 a[FA][BM * BK];           // A slices, one per ring entry
    uint64_t bfull[2], bempty[2], afull[FA], aempty[FA];
    uint64_t lfull[kLevels], lempty[kLevels];
    uint64_t drain;
    uint32_t tmem;
    int fail;
};

struct F64Args {
    int M, N;                // real accumulator rows (A side) and columns (B side)
    int nbo, mblocks, nblocks, ksteps, splits;
    long long ntiles;        // mblocks * nblocks * nbo * splits
    int a_bcast, b_bcast;
    long long Ktot;          // slice segment length
    const int* eA;           // row exponent fields [bo][RpA], [bo][RpB]
    const int* eB;
    int RpA, RpB;
    double* C;               // output, or float64 partials when splits > 1
    long long crs, ccs, cbs;
    double alpha, beta;
    int* err;
};

struct F64Coord {
    int m0, n0, bo, split, k_lo, nk;
};

__device__ __forceinline__ F64Coord f64_coord(const F64Args& a, long long t) {
    F64Coord c;
    const int nbk = (int)(t % a.nblocks);
    long long r = t / a.nblocks;
    const int mbk = (int)(r % a.mblocks);
    r /= a.mblocks;
    c.bo = (int)(r / a.splits);
    c.split = (int)(r % a.splits);
    c.m0 = mbk * BM;
    c.n0 = nbk * FN;
    const int chunk = (a.ksteps + a.splits - 1) / a.splits;
    c.k_lo = c.split * chunk;
    c.nk = max(0, min(a.ksteps, c.k_lo + chunk) - c.k_lo);
    return c;
}

// K steps per exact chunk of level q + 2: (l - 1) 64 c <= 1024.
__device__ __forceinline__ int f64_chunk_steps(int q) { return 16 / (q + 1); }

__global__ void __launch_bounds__(kF64Threads, 1)
    k_gemm_f64s(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const F64Args args) {
    extern __shared__ __align__(1024) unsigned char f64_raw[];
    F64Smem& sm = *reinterpret_cast<F64Smem*>((reinterpret_cast<uintptr_t>(f64_raw) + 1023) &
                                              ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* fail = &sm.fail;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sm.bfull[s], 1);
            mbar_init(&sm.bempty[s], 1);
        }
        for (int s = 0; s < FA; ++s) {
            mbar_init(&sm.afull[s], 1);
            mbar_init(&sm.aempty[s], 1);
        }
        for (int q = 0; q < kLevels; ++q) {
            mbar_init(&sm.lfull[q], 1);
            mbar_init(&sm.lempty[q], kF64EpiWarps);
        }
        mbar_init(&sm.drain, 1);
        sm.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sm.tmem;
    const long long Kt = args.Ktot;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            long long bit = 0, ait = 0;
            long long blast[2] = {-1, -1}, alast[FA];
            for (int s = 0; s < FA; ++s) alast[s] = -1;
            for (long long t = blockIdx.x; t < args.ntiles && !*fail; t += gridDim.x) {
                const F64Coord c = f64_coord(args, t);
                const int ba = args.a_bcast ? 0 : c.bo, bb = args.b_bcast ? 0 : c.bo;
                bool ok = true;
                for (int i = 0; i < c.nk && ok; ++i) {
                    const int kc = (c.k_lo + i) * BK;
                    const int bs = (int)(bit & 1);
                    if (bit >= 2 && !mbar_wait_or_fail(&sm.bempty[bs], (uint32_t)(((bit >> 1) - 1) & 1), fail)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&sm.bfull[bs], (uint32_t)(kSlices * FN * BK * 2));
                    for (int u = 1; u <= kSlices; ++u)   // slice u sits in segment 8 - u
                        tma_load_3d(sm.b[bs][u - 1], &tmB, &sm.bfull[bs],
                                    (int)((kSlices - u) * Kt) + kc, c.n0, bb);
                    blast[bs] = bit++;
                    for (int ts = 1; ts <= kSlices; ++ts) {
                        const int as = (int)(ait % FA);
                        if (ait >= FA && !mbar_wait_or_fail(&sm.aempty[as], (uint32_t)(((ait / FA) - 1) & 1), fail)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&sm.afull[as], (uint32_t)(BM * BK * 2));
                        tma_load_3d(sm.a[as], &tmA, &sm.afull[as], (int)((ts - 1) * Kt) + kc, c.m0, ba);
                        alast[as] = ait++;
                    }
                }
                if (!ok) break;
            }
            // Every load issued has landed before the CTA exits.
            for (int s = 0; s < 2; ++s)
                if (blast[s] >= 0) mbar_wait(&sm.bfull[s], (uint32_t)((blast[s] >> 1) & 1));
            for (int s = 0; s < FA; ++s)
                if (alast[s] >= 0) mbar_wait(&sm.afull[s], (uint32_t)((alast[s] / FA) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer.  The loops over the 36 digit pairs are unrolled and
            // the shared-memory descriptors are stepped by constants: the
            // start-address field counts 16-byte units, A ring slots are
            // BM * BK * 2 bytes apart, B slices FN * BK * 2, B buffers 8 B
            // slices, and a K sub-step of UK bf16 moves UK * 2 bytes.  (With the
            // descriptors rebuilt for every MMA, the issuing thread spent about
            // 130 cycles per 128 x 64 x 16 MMA, measured on GB300, where the
            // tensor pipe at its peak takes about 45.)
            const uint32_t idesc = instr_desc(BM, FN);
            const uint64_t a0 = smem_desc(smem_u32(sm.a[0]));
            const uint64_t b0 = smem_desc(smem_u32(sm.b[0][0]));
            constexpr uint64_t kAStep = (uint64_t)(BM * BK * 2) >> 4;
            constexpr uint64_t kBSlice = (uint64_t)(FN * BK * 2) >> 4;
            constexpr uint64_t kKStep = (uint64_t)(UK * 2) >> 4;
            long long bit = 0, ait = 0;
            // Per level q (bit q): usedm = a chunk has been started before
            // (its successor waits for the drain), parm = parity of the next
            // lempty wait.
            unsigned usedm = 0, parm = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < args.ntiles && ok && !*fail; t += gridDim.x) {
                const F64Coord c = f64_coord(args, t);
                int cnt[kLevels];
#pragma unroll
                for (int q = 0; q < kLevels; ++q) cnt[q] = 0;
                for (int i = 0; i < c.nk && ok; ++i) {
                    const int bs = (int)(bit & 1);
                    if (!mbar_wait_or_fail(&sm.bfull[bs], (uint32_t)((bit >> 1) & 1), fail)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    unsigned startedm = 0;
#pragma unroll
                    for (int q = 0; q < kLevels; ++q)
                        if (cnt[q] > 0) startedm |= 1u << q;
                    const uint64_t bbase = b0 + (uint64_t)bs * (kSlices * kBSlice);
#pragma unroll
                    for (int ts = 1; ts <= kSlices; ++ts) {
                        const int as = (int)(ait % FA);
                        if (!mbar_wait_or_fail(&sm.afull[as], (uint32_t)((ait / FA) & 1), fail)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const uint64_t ad = a0 + (uint64_t)as * kAStep;
#pragma unroll
                        for (int u = 1; u <= kSlices + 1 - ts; ++u) {
                            const int q = ts + u - 2;
                            const unsigned qb = 1u << q;
                            const uint32_t acc0 = (startedm >> q) & 1u;
                            if (!acc0) {
                                // a new chunk: the previous one has been drained
                                if (usedm & qb) {
                                    if (!mbar_wait_or_fail(&sm.lempty[q], (parm >> q) & 1u, fail)) {
                                        ok = false;
                                        break;
                                    }
                                    parm ^= qb;
                                }
                                usedm |= qb;
                                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                            }
                            const uint64_t bd = bbase + (uint64_t)(u - 1) * kBSlice;
                            const uint32_t dst = tmem + (uint32_t)(q * FN);
#pragma unroll
                            for (int kk = 0; kk < BK / UK; ++kk)
                                mma_bf16(dst, ad + kk * kKStep, bd + kk * kKStep, idesc,
                                         kk > 0 ? 1u : acc0);
                            startedm |= qb;
                        }
                        if (!ok) break;
                        mma_commit(&sm.aempty[as]);
                        ++ait;
                    }
                    if (!ok) break;
                    mma_commit(&sm.bempty[bs]);
                    ++bit;
#pragma unroll
                    for (int q = 0; q < kLevels; ++q) {
                        ++cnt[q];
                        if (cnt[q] == f64_chunk_steps(q) || i == c.nk - 1) {
                            mma_commit(&sm.lfull[q]);
                            cnt[q] = 0;
                        }
                    }
                }
            }
            // All MMAs issued have completed before TMEM is freed.
            mma_commit(&sm.drain);
            mbar_wait(&sm.drain, 0);
        }
    } else {
        // Epilogue: drains and the float64 combination of the tile.
        const int q4 = warp & 3, half = (warp - 2) >> 2;
        unsigned dpar = 0;   // bit q: parity of the next lfull wait of level q
        for (long long t = blockIdx.x; t < args.ntiles; t += gridDim.x) {
            const F64Coord c = f64_coord(args, t);
            long long H[32];
            float T[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                H[j] = 0;
                T[j] = 0.f;
            }
            int cnt[kLevels];
#pragma unroll
            for (int q = 0; q < kLevels; ++q) cnt[q] = 0;
            bool ok = true;
            for (int i = 0; i < c.nk && ok; ++i) {
#pragma unroll
                for (int q = 0; q < kLevels; ++q) {
                    ++cnt[q];
                    if (!ok || (cnt[q] != f64_chunk_steps(q) && i != c.nk - 1)) continue;
                    cnt[q] = 0;
                    if (!mbar_wait_or_fail(&sm.lfull[q], (dpar >> q) & 1u, fail)) {
                        ok = false;
                        continue;
                    }
                    dpar ^= 1u << q;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    uint32_t r[32];
                    const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) +
                                           (uint32_t)(q * FN + half * 32);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32"
                        " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
                          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
                          "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.lempty[q]);
                    const int l = q + 2;
                    if (l <= 6) {
                        const int sh = 7 * (6 - l);
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            H[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
                    } else {
                        const float w = l == 7 ? 1.f : (l == 8 ? 0.0078125f : 0.00006103515625f);
#pragma unroll
                        for (int j = 0; j < 32; ++j) T[j] = fmaf(__uint_as_float(r[j]), w, T[j]);
                    }
                }
            }
            if (!ok) break;
            // C(i, j) = alpha 2^(e_r + e_c - 42) (H + 2^-7 T) [+ beta C]
            const int i = c.m0 + q4 * 32 + lane;
            if (i >= args.M) continue;
            const int fa = args.eA[(long long)(args.a_bcast ? 0 : c.bo) * args.RpA + i];
            const int* eb = args.eB + (long long)(args.b_bcast ? 0 : c.bo) * args.RpB;
            double* Cb = args.C + (long long)c.bo * args.cbs +
                         (args.splits > 1 ? (long long)c.split * args.nbo * args.cbs : 0) +
                         (long long)i * args.crs;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = c.n0 + half * 32 + j;
                if (col >= args.N) continue;
                const int fb = eb[col];
                double v = 0.0;
                if (fa > 0 && fb > 0)
                    v = fma((double)T[j], 0.0078125, (double)H[j]) *
                        pow2((fa - 1022) + (fb - 1022) - 42);
                double* p = Cb + (long long)col * args.ccs;
                if (args.splits > 1) *p = v;
                else *p = (args.beta != 0.0 ? args.beta * *p : 0.0) + args.alpha * v;
            }
        }
    }
    __syncthreads();
    if (sm.fail && threadIdx.x == 0) atomicExch(args.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(512));
}

// C = beta C + alpha sum_split part[split] (float64 split-K partials of the
// fused kernel, in accumulator orientation: element (b, i, j) at
// part[(split nbo + b) M N + i N + j]).
__global__ void k_f64_splitsum(const double* part, int splits, int nbo, int M, int N, double* C,
                               long long crs, long long ccs, long long cbs, double alpha,
                               double beta) {
    const long long MN = (long long)M * N, tot = MN * nbo;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / MN);
        const long long r = e % MN;
        const int i = (int)(r / N), j = (int)(r % N);
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += part[(long long)sp * tot + e];
        double* p = C + (long long)b * cbs + (long long)i * crs + (long long)j * ccs;
        *p = (beta != 0.0 ? beta * *p : 0.0) + alpha * s;
    }
}

}  // namespace

namespace {

// Workspace a product takes in one piece: slices, exponents, and the slice
// row pitch (which must fit a 32-bit coordinate).
struct F64Need {
    long long slices, expo, pitch;
};

F64Need f64_need(const Gemm<double>& g) {
    const bool swap = g.N > g.M;
    const int Mr = swap ? g.N : g.M, Nr = swap ? g.M : g.N;
    const long long Kp = rup(std::max(g.K, 1), BK);
    const int nb = g.batch;
    const int nbo = g.reduce ? 1 : nb;
    const long long Ktot = g.reduce ? Kp * nb : Kp;
    const long long RpA = rup(Mr, BM), RpB = rup(Nr, FN);
    const long long sa = swap ? g.sBb : g.sAb, sb = swap ? g.sAb : g.sBb;
    const bool a_bc = !g.reduce && nb > 1 && sa == 0;
    const bool b_bc = !g.reduce && nb > 1 && sb == 0;
    const long long nba = a_bc ? 1 : nbo, nbb = b_bc ? 1 : nbo;
    const long long pitch = kSlices * Ktot;
    return F64Need{(RpA * nba + RpB * nbb) * pitch, RpA * nba + RpB * nbb, pitch};
}

bool f64_fits(const Gemm<double>& g, const F64TcWorkspace& ws) {
    const F64Need n = f64_need(g);
    return (size_t)n.slices <= ws.slice_elems && (size_t)n.expo <= ws.expo_elems &&
           n.pitch <= INT32_MAX;
}

cudaError_t gemm_f64_tc_one(const Gemm<double>& g, const F64TcWorkspace& ws, cudaStream_t s);

}  // namespace

// A product whose slices do not fit the workspace is cut into pieces that
// do: batches first (a batch-reduced product accumulates its later pieces
// into C with beta = 1), then the rows or the columns of C, whichever are
// more, in halves rounded to the 128-row tile.
cudaError_t gemm_f64_tc(const Gemm<double>& g, const F64TcWorkspace& ws, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    if (f64_fits(g, ws)) return gemm_f64_tc_one(g, ws, s);
    Gemm<double> g1 = g, g2 = g;
    if (g.batch > 1) {
        const int b1 = g.batch / 2;
        g1.batch = b1;
        g2.batch = g.batch - b1;
        g2.A.p = g.A.p + (long long)b1 * g.sAb;
        g2.B.p = g.B.p + (long long)b1 * g.sBb;
        if (g.reduce) {
            g2.beta = 1.0;
        } else {
            g2.C = g.C + (long long)b1 * g.sCb;
        }
    } else if (g.M >= g.N && g.M > BM) {
        const int m1 = (int)rup((g.M + 1) / 2, BM);
        g1.M = m1;
        g2.M = g.M - m1;
        g2.A.p = g.A.p + (long long)m1 * g.A.rs;
        g2.C = g.C + (long long)m1 * g.ldc;
    } else if (g.N > BM) {
        const int n1 = (int)rup((g.N + 1) / 2, BM);
        g1.N = n1;
        g2.N = g.N - n1;
        g2.B.p = g.B.p + (long long)n1 * g.B.cs;
        g2.C = g.C + n1;
    } else {
        return cudaErrorMemoryAllocation;   // a single tile row and column do not fit
    }
    cudaError_t e = gemm_f64_tc(g1, ws, s);
    if (e != cudaSuccess) return e;
    return gemm_f64_tc(g2, ws, s);
}

namespace {

cudaError_t gemm_f64_tc_one(const Gemm<double>& g, const F64TcWorkspace& ws, cudaStream_t s) {
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    const bool swap = g.N > g.M;
    const int Mr = swap ? g.N : g.M, Nr = swap ? g.M : g.N;
    const long long Kp = rup(std::max(g.K, 1), BK);
    const int nb = g.batch;
    const int nbo = g.reduce ? 1 : nb;
    const long long Ktot = g.reduce ? Kp * nb : Kp;
    const long long RpA = rup(Mr, BM), RpB = rup(Nr, FN);
    View<double> va = g.A, vb{g.B.p, g.B.cs, g.B.rs};
    long long sa = g.sAb, sb = g.sBb;
    if (swap) {
        std::swap(va, vb);
        std::swap(sa, sb);
    }
    const bool a_bc = !g.reduce && nb > 1 && sa == 0;
    const bool b_bc = !g.reduce && nb > 1 && sb == 0;
    const int nba = a_bc ? 1 : nbo, nbb = b_bc ? 1 : nbo;
    const long long pitch = kSlices * Ktot;
    const long long sliceA = RpA * pitch * nba, sliceB = RpB * pitch * nbb;
    if ((size_t)(sliceA + sliceB) > ws.slice_elems) return cudaErrorMemoryAllocation;
    if ((size_t)(RpA * nba + RpB * nbb) > ws.expo_elems) return cudaErrorMemoryAllocation;
    if (pitch > INT32_MAX) return cudaErrorMemoryAllocation;
    const int mblocks = (int)(RpA / BM), nblocks = (int)(RpB / FN);
    const long long tiles = (long long)mblocks * nblocks * nbo;
    const int ksteps = (int)(Ktot / BK);
    const long long sms = device_sms();
    // Split K so that the work items fill whole waves of SMs: the split
    // count (at most 32, at least 8 K steps each) with the best ratio of
    // items to SM slots in the waves they take; the float64 partials of the
    // splits go to the workspace's partial buffer.
    int splits = 1;
    {
        const long long per = (long long)Mr * Nr * nbo;
        auto fill = [&](long long sp) {
            const long long items = tiles * sp;
            return (double)items / (double)(((items + sms - 1) / sms) * sms);
        };
        double best = fill(1);
        for (int sp = 2; sp <= 32 && ksteps / sp >= 8; ++sp) {
            if ((size_t)(per * sp) > ws.part_elems / 2) break;
            const double f = fill(sp);
            if (f > best + 0.02) {
                best = f;
                splits = sp;
            }
        }
    }

    __nv_bfloat16* slA = ws.slices;
    __nv_bfloat16* slB = ws.slices + sliceA;
    int* eA = ws.expo;
    int* eB = ws.expo + RpA * nba;
    // Row exponents and slices of both operands.
    const int red = g.reduce ? 1 : 0;
    if ((e = cudaMemsetAsync(ws.expo, 0, sizeof(int) * (RpA * nba + RpB * nbb), s)) !=
        cudaSuccess)
        return e;
    struct Side { View<double> v; long long sbat; int R; long long Rp; int nbg; __nv_bfloat16* sl;
                  int* ex; int rev; };
    const Side sides[2] = {{va, sa, Mr, RpA, a_bc ? 1 : nb, slA, eA, 0},
                           {vb, sb, Nr, RpB, b_bc ? 1 : nb, slB, eB, 1}};
    for (const Side& sd : sides) {
        const dim3 grid(cdiv(Kp, PK_K), std::min<unsigned>(cdiv(sd.Rp, PK_R), 65535), sd.nbg);
        k_row_exp<<<grid, 256, 0, s>>>(sd.v.p, sd.v.rs, sd.v.cs, sd.sbat, sd.R, g.K, (int)sd.Rp,
                                       red, sd.ex);
        k_slice64<<<grid, 256, 0, s>>>(sd.v.p, sd.v.rs, sd.v.cs, sd.sbat, sd.R, g.K, nb,
                                       (int)sd.Rp, (int)Kp, red, sd.rev, sd.ex, sd.sl);
        count_launches(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    CUtensorMap mA, mB;
    if ((e = make_map_pitch(&mA, slA, pitch, pitch, RpA, nba, BM)) != cudaSuccess) return e;
    if ((e = make_map_pitch(&mB, slB, pitch, pitch, RpB, nbb, FN)) != cudaSuccess) return e;
    F64Args a{};
    a.M = Mr;
    a.N = Nr;
    a.nbo = nbo;
    a.mblocks = mblocks;
    a.nblocks = nblocks;
    a.ksteps = ksteps;
    a.splits = splits;
    a.ntiles = tiles * splits;
    a.a_bcast = a_bc ? 1 : 0;
    a.b_bcast = b_bc ? 1 : 0;
    a.Ktot = Ktot;
    a.eA = eA;
    a.eB = eB;
    a.RpA = (int)RpA;
    a.RpB = (int)RpB;
    a.alpha = g.alpha;
    a.beta = g.beta;
    a.err = ws.err;
    // accumulator (i, j) is C's (m, n), or (n, m) when the operands were swapped
    const long long crs = swap ? 1 : g.ldc, ccs = swap ? g.ldc : 1;
    const long long cbs = g.reduce ? 0 : g.sCb;
    double* part = reinterpret_cast<double*>(ws.part);
    if (splits > 1) {
        a.C = part;
        a.crs = Nr;
        a.ccs = 1;
        a.cbs = (long long)Mr * Nr;
    } else {
        a.C = g.C;
        a.crs = crs;
        a.ccs = ccs;
        a.cbs = cbs;
    }
    const int smem = (int)sizeof(F64Smem) + 1024;
    if ((e = smem_optin((const void*)k_gemm_f64s, smem)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<long long>(a.ntiles, sms);
    k_gemm_f64s<<<grid, kF64Threads, smem, s>>>(mA, mB, a);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (splits > 1) {
        const long long tot = (long long)Mr * Nr * nbo;
        const unsigned blocks = (unsigned)std::min<long long>((tot + 255) / 256, sms * 16);
        k_f64_splitsum<<<blocks, 256, 0, s>>>(part, splits, nbo, Mr, Nr, g.C, crs, ccs, cbs,
                                              g.alpha, g.beta);
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

// ---------------------------------------------------------------------------
// Randomised self-test: tensor-core products against the CUDA-core products
// of the same float32 operands over random shapes, orientations, batch modes
// (separate, shared operand, batch-reduced), split-K and beta.
namespace {

unsigned long long st_next(unsigned long long& s) {
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    return s;
}

__global__ void k_fill_uniform(float* p, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        p[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 0.5f;
    }
}

__global__ void k_max_abs_diff(const float* a, const float* b, long long n, float* out) {
    float m = 0.f, s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        m = fmaxf(m, fabsf(a[i] - b[i]));
        s = fmaxf(s, fabsf(b[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
        s = fmaxf(s, __shfl_down_sync(0xffffffffu, s, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
        atomicMax(reinterpret_cast<int*>(out + 1), __float_as_int(s));
    }
}

}  // namespace

cudaError_t gemm_tc_selftest(int cases, unsigned long long seed, double* max_rel,
                             int* failures, cudaStream_t st) {
    *max_rel = 0;
    *failures = 0;
    const long long cap = 1LL << 22;   // elements per operand buffer
    float *A = nullptr, *B = nullptr, *C1 = nullptr, *C2 = nullptr, *red = nullptr, *simt = nullptr;
    TcWorkspace ws{};
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void**)&A, cap * 4);
    al((void**)&B, cap * 4);
    al((void**)&C1, cap * 4);
    al((void**)&C2, cap * 4);
    al((void**)&red, 8);
    al((void**)&simt, cap * 4);
    ws.elems = (size_t)1 << 25;
    al((void**)&ws.buf, ws.elems * 2);
    ws.partial_elems = (size_t)1 << 24;
    al((void**)&ws.partial, ws.partial_elems * 4);
    al((void**)&ws.err, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.err, 0, 4, st);
    unsigned long long s = seed * 2654435761ULL + 1;
    for (int c = 0; c < cases && e == cudaSuccess; ++c) {
        Gemm<float> g;
        g.M = 1 + (int)(st_next(s) % 700);
        g.N = 1 + (int)(st_next(s) % 700);
        g.K = 1 + (int)(st_next(s) % 900);
        g.batch = 1 + (int)(st_next(s) % 4);
        const int mode = (int)(st_next(s) % 4);   // 0 separate, 1 shared A, 2 shared B, 3 reduce
        g.reduce = mode == 3 && g.batch > 1;
        const bool ta = st_next(s) & 1, tb = st_next(s) & 1;
        const int nprod = (st_next(s) % 3 == 0) ? 1 : 3;
        g.beta = (st_next(s) & 1) ? 0.5 : 0.0;
        // a general alpha and powers of two
        g.alpha = (c & 1) ? 1.25 : ((c & 2) ? -0.5 : 2.0);
        while ((long long)g.batch * g.M * g.K > cap || (long long)g.batch * g.K * g.N > cap ||
               (long long)g.batch * g.M * g.N > cap)
            g.K = std::max(1, g.K / 2), g.M = std::max(1, g.M * 3 / 4);
        const long long sa = (long long)g.M * g.K, sb = (long long)g.K * g.N,
                        sc = (long long)g.M * g.N;
        g.A = ta ? View<float>{A, 1, g.M} : View<float>{A, g.K, 1};
        g.B = tb ? View<float>{B, 1, g.K} : View<float>{B, g.N, 1};
        g.sAb = mode == 1 ? 0 : sa;
        g.sBb = mode == 2 ? 0 : sb;
        g.ldc = g.N;
        g.sCb = sc;
        const long long nC = (g.reduce ? 1 : g.batch) * sc;
        k_fill_uniform<<<256, 256, 0, st>>>(A, g.batch * sa, st_next(s));
        k_fill_uniform<<<256, 256, 0, st>>>(B, g.batch * sb, st_next(s));
        k_fill_uniform<<<256, 256, 0, st>>>(C1, nC, st_next(s));
        count_launches(3);
        if ((e = cudaMemcpyAsync(C2, C1, nC * 4, cudaMemcpyDeviceToDevice, st))) break;
        Gemm<float> h = g;
        g.C = C1;
        h.C = C2;
        h.ws = simt;
        h.ws_elems = cap;
        if ((e = gemm_tc(g, ws, nprod, st))) break;
        if ((e = gemm_simt(h, st))) break;
        if ((e = cudaMemsetAsync(red, 0, 8, st))) break;
        k_max_abs_diff<<<256, 256, 0, st>>>(C1, C2, nC, red);
        count_launches(1);
        float hr[2] = {0, 0};
        int herr = 0;
        if ((e = cudaMemcpyAsync(hr, red, 8, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaMemcpyAsync(&herr, ws.err, 4, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        // bf16x3: about 3 x 2^-17 per product, float32 sums over K terms;
        // bf16x1: 2^-8 per factor
        const double scale = std::max(1.0f, hr[1]);
        const double rel = hr[0] / scale;
        const double bound = (nprod == 3 ? 2e-5 : 2e-2) * std::sqrt((double)g.K + 1) *
                             (g.reduce ? std::sqrt((double)g.batch) : 1.0);
        *max_rel = std::max(*max_rel, nprod == 3 ? rel : 0.0);
        if (herr || !(rel <= bound)) ++*failures;
    }
    for (void* p : {(void*)A, (void*)B, (void*)C1, (void*)C2, (void*)red, (void*)simt,
                    (void*)ws.buf, (void*)ws.partial, (void*)ws.err})
        if (p) cudaFree(p);
    return e;
}

namespace {

__global__ void k_fill_uniform64(double* p, long long n, unsigned long long seed, int spread) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        double v = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        // spread > 0: magnitudes over 2^-spread .. 1 (rows with a wide range)
        if (spread > 0) v = scalbn(v, -(int)((z >> 3) % (unsigned long long)(spread + 1)));
        p[i] = v;
    }
}

__global__ void k_max_abs_diff64(const double* a, const double* b, long long n, double* out) {
    double m = 0.0, s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        m = fmax(m, fabs(a[i] - b[i]));
        s = fmax(s, fabs(b[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
        atomicMax(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)__double_as_longlong(s));
    }
}

}  // namespace

cudaError_t gemm_f64_tc_selftest(int cases, unsigned long long seed, double* max_rel,
                                 int* failures, cudaStream_t st) {
    *max_rel = 0;
    *failures = 0;
    const long long cap = 1LL << 21;   // elements per operand buffer
    double *A = nullptr, *B = nullptr, *C1 = nullptr, *C2 = nullptr, *red = nullptr, *simt = nullptr;
    F64TcWorkspace ws{};
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void**)&A, cap * 8);
    al((void**)&B, cap * 8);
    al((void**)&C1, cap * 8);
    al((void**)&C2, cap * 8);
    al((void**)&red, 16);
    al((void**)&simt, cap * 8);
    ws.slice_elems = (size_t)1 << 26;
    al((void**)&ws.slices, ws.slice_elems * 2);
    ws.part_elems = (size_t)1 << 28;   // the 8 levels of the largest case (about 1.4e8)
    al((void**)&ws.part, ws.part_elems * 4);
    ws.expo_elems = (size_t)1 << 16;
    al((void**)&ws.expo, ws.expo_elems * 4);
    al((void**)&ws.err, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.err, 0, 4, st);
    unsigned long long s = seed * 2654435761ULL + 7;
    for (int c = 0; c < cases && e == cudaSuccess; ++c) {
        Gemm<double> g;
        g.M = 1 + (int)(st_next(s) % 600);
        g.N = 1 + (int)(st_next(s) % 600);
        g.K = 1 + (int)(st_next(s) % 2600);    // up to three exact K chunks
        g.batch = 1 + (int)(st_next(s) % 4);
        const int mode = (int)(st_next(s) % 4);   // 0 separate, 1 shared A, 2 shared B, 3 reduce
        g.reduce = mode == 3 && g.batch > 1;
        const bool ta = st_next(s) & 1, tb = st_next(s) & 1;
        const int spread = (st_next(s) % 3 == 0) ? 40 : 0;
        g.beta = (st_next(s) & 1) ? 0.5 : 0.0;
        // a general alpha and powers of two
        g.alpha = (c & 1) ? 1.25 : ((c & 2) ? -0.5 : 2.0);
        while ((long long)g.batch * g.M * g.K > cap || (long long)g.batch * g.K * g.N > cap ||
               (long long)g.batch * g.M * g.N > cap)
            g.K = std::max(1, g.K / 2), g.M = std::max(1, g.M * 3 / 4);
        const long long sa = (long long)g.M * g.K, sb = (long long)g.K * g.N,
                        sc = (long long)g.M * g.N;
        g.A = ta ? View<double>{A, 1, g.M} : View<double>{A, g.K, 1};
        g.B = tb ? View<double>{B, 1, g.K} : View<double>{B, g.N, 1};
        g.sAb = mode == 1 ? 0 : sa;
        g.sBb = mode == 2 ? 0 : sb;
        g.ldc = g.N;
        g.sCb = sc;
        const long long nC = (g.reduce ? 1 : g.batch) * sc;
        k_fill_uniform64<<<256, 256, 0, st>>>(A, g.batch * sa, st_next(s), spread);
        k_fill_uniform64<<<256, 256, 0, st>>>(B, g.batch * sb, st_next(s), spread);
        k_fill_uniform64<<<256, 256, 0, st>>>(C1, nC, st_next(s), 0);
        count_launches(3);
        if ((e = cudaMemcpyAsync(C2, C1, nC * 8, cudaMemcpyDeviceToDevice, st))) break;
        Gemm<double> h = g;
        g.C = C1;
        h.C = C2;
        h.ws = simt;
        h.ws_elems = cap;
        // Every third case gets a third of the slice workspace it needs, so
        // that the product is cut into pieces.
        F64TcWorkspace wsc = ws;
        if (c % 3 == 2) {
            const long long Kp = rup(std::max(g.K, 1), BK);
            wsc.slice_elems = (size_t)std::max<long long>(f64_need(g).slices / 3,
                                                          2LL * BM * kSlices * Kp);
        }
        if ((e = gemm_f64_tc(g, wsc, st))) break;
        if ((e = gemm_simt(h, st))) break;
        if ((e = cudaMemsetAsync(red, 0, 16, st))) break;
        k_max_abs_diff64<<<256, 256, 0, st>>>(C1, C2, nC, red);
        count_launches(1);
        double hr[2] = {0, 0};
        int herr = 0;
        if ((e = cudaMemcpyAsync(hr, red, 16, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaMemcpyAsync(&herr, ws.err, 4, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        // Both sides are float64-accurate: a few units of 2^-53 times the
        // size of the sums (K terms of up to 1/4, and beta C).
        const double scale = std::max(1.0, hr[1]);
        const double rel = hr[0] / scale;
        const double bound = 1e-15 * ((double)g.K * (g.reduce ? g.batch : 1) + 1);
        *max_rel = std::max(*max_rel, rel);
        if (herr || !(rel <= bound)) ++*failures;
    }
    for (void* p : {(void*)A, (void*)B, (void*)C1, (void*)C2, (void*)red, (void*)simt,
                    (void*)ws.slices, (void*)ws.part, (void*)ws.expo, (void*)ws.err})
        if (p) cudaFree(p);
    return e;
}

}  // namespace thc
