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
#include <mutex>

#include "common.cuh"
#include "gemm_tc.cuh"

namespace thc {
namespace {

constexpr int BM = 128;          // UMMA M (rows of the accumulator)
constexpr int BK = 64;           // K per stage: one 128-byte swizzle atom of bf16
constexpr int UK = 16;           // K per tcgen05.mma for 16-bit inputs
constexpr int STAGES = 3;
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

template <int BN>
struct TcSmem {
    __nv_bfloat16 a_hi[STAGES][BM * BK];
    __nv_bfloat16 a_lo[STAGES][BM * BK];
    __nv_bfloat16 b_hi[STAGES][BN * BK];
    __nv_bfloat16 b_lo[STAGES][BN * BK];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t done;
    uint32_t tmem;
    int fail;
};

struct TcArgs {
    int M, N;              // real accumulator rows (UMMA M side) and columns
    int nbo;               // output batches
    int ksteps;            // 64-wide K steps per output batch
    int splits;
    float* C;              // output (or partials when splits > 1)
    long long crs, ccs, cbs;   // C(i, j) of batch b at C[b*cbs + i*crs + j*ccs]
    float alpha, beta;
    int nprod;
    int a_bcast, b_bcast;  // operand shared by every batch: packed once, batch coord 0
    int* err;
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              const TcArgs args) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    // 1024-byte alignment of the tile ring (required by the 128-byte swizzle)
    TcSmem<BN>& sm = *reinterpret_cast<TcSmem<BN>*>(
        (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int bo = blockIdx.z / args.splits, split = blockIdx.z % args.splits;
    const int chunk = (args.ksteps + args.splits - 1) / args.splits;
    const int k_lo = split * chunk, k_hi = min(args.ksteps, k_lo + chunk);
    const int nk = max(0, k_hi - k_lo);
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        mbar_init(&sm.done, 1);
        sm.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {
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

    if (warp == 0 && lane == 0 && nk > 0) {
        // TMA producer
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            if (i >= STAGES && !mbar_wait(&sm.empty[s], ((i / STAGES) - 1) & 1)) {
                atomicExch(&sm.fail, 1);
                break;
            }
            if (sm.fail) break;
            const int kc = (k_lo + i) * BK;
            mbar_expect_tx(&sm.full[s], stage_bytes);
            const int ba = args.a_bcast ? 0 : bo, bb = args.b_bcast ? 0 : bo;
            tma_load_3d(sm.a_hi[s], &ta_hi, &sm.full[s], kc, m0, ba);
            tma_load_3d(sm.b_hi[s], &tb_hi, &sm.full[s], kc, n0, bb);
            if (args.nprod == 3) {
                tma_load_3d(sm.a_lo[s], &ta_lo, &sm.full[s], kc, m0, ba);
                tma_load_3d(sm.b_lo[s], &tb_lo, &sm.full[s], kc, n0, bb);
            }
        }
    } else if (warp == 1 && lane == 0 && nk > 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(BM, BN);
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            if (!mbar_wait(&sm.full[s], (i / STAGES) & 1)) {
                atomicExch(&sm.fail, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t ah = smem_u32(sm.a_hi[s]), bh = smem_u32(sm.b_hi[s]);
            const uint32_t al = smem_u32(sm.a_lo[s]), bl = smem_u32(sm.b_lo[s]);
#pragma unroll
            for (int kk = 0; kk < BK / UK; ++kk) {
                const uint32_t off = kk * UK * 2;   // bytes along K inside the swizzle atom
                const uint32_t acc0 = (i > 0 || kk > 0) ? 1u : 0u;
                mma_bf16(tmem, smem_desc(ah + off), smem_desc(bh + off), idesc, acc0);
                if (args.nprod == 3) {
                    mma_bf16(tmem, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
                    mma_bf16(tmem, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
                }
            }
            mma_commit(&sm.empty[s]);
        }
        mma_commit(&sm.done);
    }
    __syncwarp();

    // Epilogue: warp w owns accumulator rows 32w .. 32w+31.
    if (nk > 0 && !mbar_wait(&sm.done, 0)) atomicExch(&sm.fail, 1);
    __syncthreads();
    const bool ok = sm.fail == 0;   // uniform across the block
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // The operand ring is idle now (every load was consumed by an MMA that
    // completed before `done`): stage the 128 x BN accumulator tile there and
    // write it out along whichever index of C is contiguous.
    float* stage = reinterpret_cast<float*>(&sm.a_hi[0][0]);
    constexpr int LDS_ = BN + 1;
    float* Cb = args.C + (long long)bo * args.cbs +
                (args.splits > 1 ? (long long)split * args.nbo * args.cbs : 0);
    if (ok) {
        const int rl = warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            if (nk > 0) {
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32"
                    " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) stage[rl * LDS_ + c0 + j] = __uint_as_float(r[j]);
        }
    }
    __syncthreads();
    if (ok) {
        auto put = [&](int i, int j, float v) {
            float* c = Cb + (long long)(m0 + i) * args.crs + (long long)(n0 + j) * args.ccs;
            if (args.splits > 1) *c = v;
            else *c = args.beta != 0.f ? fmaf(args.beta, *c, args.alpha * v) : args.alpha * v;
        };
        if (args.ccs == 1) {
            for (int i = warp; i < BM; i += 4) {
                if (m0 + i >= args.M) break;
                for (int j = lane; j < BN; j += 32)
                    if (n0 + j < args.N) put(i, j, stage[i * LDS_ + j]);
            }
        } else {
            for (int j = warp; j < BN; j += 4) {
                if (n0 + j >= args.N) break;
                for (int i = lane; i < BM; i += 32)
                    if (m0 + i < args.M) put(i, j, stage[i * LDS_ + j]);
            }
        }
    }
    if (!ok && threadIdx.x == 0) atomicExch(args.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kCols));
}

// Pack a strided float32 operand into bf16 hi/lo, K-major, padded:
// out[bo][r][kb*Kp + k] = split(src(b, r, k)), r < Rp, k < Kp, with
// (bo, kb) = (b, 0) for batched products and (0, b) for batch-reduced ones.
__global__ void k_pack(const float* src, long long rs, long long ks, long long bs, int R,
                       int Kd, int nb, int Rp, int Kp, int reduce, __nv_bfloat16* hi,
                       __nv_bfloat16* lo) {
    __shared__ float tile[32][33];
    const int b = blockIdx.z;
    const int k0 = blockIdx.x * 32;
    const float* s = src + (long long)b * bs;
    const bool kfast = ks <= rs;
    const long long Ktot = reduce ? (long long)nb * Kp : Kp;
    const int bo = reduce ? 0 : b, kb = reduce ? b : 0;
    for (int r0 = blockIdx.y * 32; r0 < Rp; r0 += gridDim.y * 32) {
        for (int j = threadIdx.y; j < 32; j += 8) {
            int r, k;
            if (kfast) { r = r0 + j; k = k0 + threadIdx.x; }
            else       { r = r0 + threadIdx.x; k = k0 + j; }
            const float v = (r < R && k < Kd) ? s[(long long)r * rs + (long long)k * ks] : 0.f;
            if (kfast) tile[j][threadIdx.x] = v;
            else tile[threadIdx.x][j] = v;
        }
        __syncthreads();
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int r = r0 + j, k = k0 + threadIdx.x;
            if (r >= Rp || k >= Kp) continue;
            const float v = tile[j][threadIdx.x];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const long long o = ((long long)bo * Rp + r) * Ktot + (long long)kb * Kp + k;
            hi[o] = h;
            if (lo) lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
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
cudaError_t launch_tc(const CUtensorMap* maps, const TcArgs& a, int mblocks, int nblocks,
                      cudaStream_t s) {
    const int smem = (int)sizeof(TcSmem<BN>) + 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(nblocks, mblocks, a.nbo * a.splits);
    k_gemm_tc<BN><<<grid, 128, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
    count_launches(1);
    return cudaGetLastError();
}

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

}  // namespace

size_t gemm_tc_pack_elems(int M, int N, int K, int batch, bool reduce) {
    // Worst case over the two orientations (both sides padded to 128).
    const long long Kp = rup(std::max(K, 1), BK);
    const long long Rm = rup(M, 128), Rn = rup(N, 128);
    return (size_t)(2 * (Rm + Rn) * Kp * batch);
}

cudaError_t gemm_tc(const Gemm<float>& g, const TcWorkspace& ws, int nprod, cudaStream_t s) {
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
    const size_t need = (nprod == 3 ? 2 : 1) * (needA + needB);
    if (need > ws.elems) return cudaErrorMemoryAllocation;
    __nv_bfloat16* a_hi = ws.buf;
    __nv_bfloat16* b_hi = a_hi + needA;
    __nv_bfloat16* a_lo = nprod == 3 ? b_hi + needB : nullptr;
    __nv_bfloat16* b_lo = nprod == 3 ? a_lo + needA : nullptr;
    {
        dim3 blk(32, 8);
        dim3 gA(cdiv(Kp, 32), std::min<unsigned>(cdiv(RpA, 32), 65535), a_bc ? 1 : nb);
        dim3 gB(cdiv(Kp, 32), std::min<unsigned>(cdiv(RpB, 32), 65535), b_bc ? 1 : nb);
        k_pack<<<gA, blk, 0, s>>>(va.p, va.rs, va.cs, sa, Mr, g.K, nb, (int)RpA, (int)Kp,
                                  g.reduce ? 1 : 0, a_hi, a_lo);
        k_pack<<<gB, blk, 0, s>>>(vb.p, vb.rs, vb.cs, sb, Nr, g.K, nb, (int)RpB, (int)Kp,
                                  g.reduce ? 1 : 0, b_hi, b_lo);
        count_launches(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
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
    if (BN == 32) e = launch_tc<32>(maps, a, mblocks, nblocks, s);
    else if (BN == 64) e = launch_tc<64>(maps, a, mblocks, nblocks, s);
    else e = launch_tc<128>(maps, a, mblocks, nblocks, s);
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

}  // namespace thc
