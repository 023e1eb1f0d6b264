// Float64-accurate triangle kernel on the FP32 pipe (Alg. 6 line 11, Eq. 34):
//   H^XYZ += sum_I (E_I^XY F_I^XZ + E_I^XZ F_I^XY) G_I^YZ.
//
// The step is not a product (every operand shares two of the three output
// indices), so it cannot use the tensor cores, and GB300's FP64 pipe delivers
// 1/64 of the FP32 rate.  Here every float64 operand is carried as an
// unevaluated sum of two floats x = x_h + x_l (x_h = fl32(x), x_l = fl32(x -
// x_h); 48 significant bits), and the arithmetic uses error-free
// transformations:
//   * TwoProduct with an FMA:  p = fl(a b),  e = fma(a, b, -p),  a b = p + e
//     exactly (Karp and Markstein; Ogita, Rump and Oishi 2005, Alg. 3.3);
//   * TwoSum (Knuth):  s = fl(a + b),  z = s - a,
//     e = (a - (s - z)) + (b - z),  a + b = s + e exactly.
// t^XYZ = E^XY F^XZ + E^XZ F^XY is formed as a float pair (th, tl) from two
// exact products of the high parts, their exact sum, and the four cross
// products of high and low parts; H accumulates t G as a float pair whose
// high word is updated by TwoSum, the rounding errors and the low-order
// product terms going to the low word.  Each term carries an error of about
// 2^-45 of |E F G| (2^-43 at worst, from the roundings of the low words;
// float64: 2^-53), far below the 1e-10 bound on the residual.
//
// Like the float64 kernel, a block takes a pair of mirror (Y, Z) tiles, since
// t is symmetric in (Y, Z): one t feeds H^XYZ (with G^YZ) and H^XZY (with
// G^ZY).  Two amplitude indices X run in the two lanes of packed f32x2
// instructions (add/sub/fma.rn.f32x2), which halves the issued
// instructions; E and F are stored with the two X rows of a pair interleaved
// ({h(x), h(x+1), l(x), l(x+1)}), so that one 16-byte load gives both lanes.
// Per (X pair, Y, Z) pair of mirror outputs: 19 packed operations for t and
// 12 for each accumulation, i.e. 21.5 float32 operations per (I, X, Y, Z) term.
#include "kernels.cuh"

namespace thc {
namespace {

typedef unsigned long long f2;   // two float32 lanes: low word = lane 0

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// -a in both lanes: a sign-bit flip on the integer pipe (the FMA pipe is the
// busy one here; -0 for a zero lane, which no later sum can tell from +0).
__device__ __forceinline__ f2 neg2(f2 a) {
#ifdef THC_DF_SUBNEG
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(0ull), "l"(a));
    return d;
#else
    return a ^ 0x8000000080000000ull;
#endif
}
// The rounded product fl(a b), written as fma(a, b, +0).  ptxas contracts a
// packed mul.rn.f32x2 whose result feeds an add.rn.f32x2 into one fused
// operation, which would round a b + c once where TwoSum needs fl(a b)
// itself (measured on GB300: every case where the two differ); an FMA with
// a zero addend is left alone.
__device__ __forceinline__ f2 prod2(f2 a, f2 b) { return fma2(a, b, 0ull); }

// t = a b + c d for float pairs a = aH + aL etc.: (th, tl) with th + tl = t
// up to the dropped low*low products and the roundings of the cross terms.
__device__ __forceinline__ void df_dot2(f2 aH, f2 aL, f2 bH, f2 bL, f2 cH, f2 cL, f2 dH,
                                        f2 dL, f2& th, f2& tl) {
    const f2 p1 = prod2(aH, bH);
    const f2 e1 = fma2(aH, bH, neg2(p1));   // aH bH - p1, exact
    const f2 p2 = prod2(cH, dH);
    const f2 e2 = fma2(cH, dH, neg2(p2));
    const f2 s = add2(p1, p2);                     // TwoSum(p1, p2)
    const f2 z = sub2(s, p1);
    const f2 es = add2(sub2(p1, sub2(s, z)), sub2(p2, z));
    f2 lo = fma2(aH, bL, e1);
    lo = fma2(aL, bH, lo);
    lo = fma2(cH, dL, lo);
    lo = fma2(cL, dH, lo);
    lo = add2(lo, e2);
    th = s;
    tl = add2(lo, es);
}

// (Sh, Sl) -= t g, with thn = -th: the accumulator holds -H so that the
// negated rounded product qn = fl(-th gH) feeds both TwoProduct and TwoSum.
__device__ __forceinline__ void df_acc(f2& Sh, f2& Sl, f2 th, f2 tl, f2 thn, f2 gH, f2 gL) {
    const f2 qn = prod2(thn, gH);      // -fl(th gH)
    const f2 e = fma2(th, gH, qn);     // th gH - fl(th gH), exact
    f2 low = fma2(th, gL, e);
    low = fma2(tl, gH, low);           // t g - fl(th gH), to second order
    const f2 s = add2(Sh, qn);         // TwoSum(Sh, qn)
    const f2 z = sub2(s, Sh);
    const f2 es = add2(sub2(Sh, sub2(s, z)), sub2(qn, z));
    Sl = sub2(add2(Sl, es), low);
    Sh = s;
}

constexpr int DX = 4;     // amplitude indices X per block (two lane pairs)
constexpr int DT = 32;    // Y and Z tile
constexpr int DS = 4;     // grid points per pipeline stage
constexpr int DTH = 256;  // threads: 16 x 16, each a 2 x 2 (Y, Z) block

static_assert(DS * 2 * DT == DTH, "one E/F element per thread and stage");
static_assert(DT * DT == 4 * DTH / 8 * 8 && DTH / DT * 4 == DT, "four G rows per thread");

struct DfStage {
    float4 ey[DS][2][DT];         // E^{x,Y} of the Y tile, {h(x), h(x+1), l(x), l(x+1)}
    float4 ez[DS][2][DT];         // E^{x,Z} of the Z tile
    float4 fy[DS][2][DT];
    float4 fz[DS][2][DT];
    float2 g1[DS][DT][DT + 1];    // {h, l} of G^YZ, rows Y
    float2 g2[DS][DT][DT + 1];    // {h, l} of G^ZY, rows Z
};

__device__ __forceinline__ void cpa16(void* dst, const void* src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cpa8(void* dst, const void* src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 8 : 0));
}

// Per-thread copy plan of the block's tiles, fixed for the whole launch.
// G tiles: thread tid copies column c = tid % 32 of rows r0 + 8 q (q < 4) of
// both tiles for each grid point of a stage; E, F: thread tid copies the
// element (s, xp, c) = (tid / 64, tid / 32 % 2, tid % 32) of the four arrays.
struct DfPlan {
    int g1off[4], g2off[4];   // (Y0 + r) P + Z0 + c, (Z0 + r) P + Y0 + c
    unsigned gok;             // bit q: g1 row in range, bit 4 + q: g2 row in range
    long long qoff;           // (xp0 + xp) P
    int cy, cz;               // Y0 + c, Z0 + c
    bool qok, yok, zok;
};

__device__ __forceinline__ DfPlan df_plan(int P, int nXp, int xp0, int Y0, int Z0) {
    DfPlan pl;
    const int tid = threadIdx.x, c = tid & 31, r0 = tid >> 5;
    pl.gok = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + 8 * q;
        pl.g1off[q] = (Y0 + r) * P + Z0 + c;
        pl.g2off[q] = (Z0 + r) * P + Y0 + c;
        if (Y0 + r < P && Z0 + c < P) pl.gok |= 1u << q;
        if (Z0 + r < P && Y0 + c < P) pl.gok |= 1u << (4 + q);
    }
    const int xp = (tid >> 5) & 1;
    pl.qoff = (long long)(xp0 + xp) * P;
    pl.qok = xp0 + xp < nXp;
    pl.cy = Y0 + c;
    pl.cz = Z0 + c;
    pl.yok = Y0 + c < P;
    pl.zok = Z0 + c < P;
    return pl;
}

// Stage grid points I0 .. I0 + DS - 1 of the block's tiles (zeros outside).
__device__ __forceinline__ void df_load(DfStage& st, const DfPlan& pl, const float4* E4,
                                        const float4* F4, const float2* G2, int P, int nXp,
                                        int nI, int I0) {
    const long long PP = (long long)P * P, XP = (long long)nXp * P;
    const int tid = threadIdx.x, c = tid & 31, r0 = tid >> 5;
#pragma unroll
    for (int s = 0; s < DS; ++s) {
        const int I = I0 + s;
        const bool iok = I < nI;
        const float2* Gi = G2 + (iok ? I * PP : 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool ok1 = iok && (pl.gok >> q & 1u);
            const bool ok2 = iok && (pl.gok >> (4 + q) & 1u);
            cpa8(&st.g1[s][r0 + 8 * q][c], ok1 ? Gi + pl.g1off[q] : G2, ok1);
            cpa8(&st.g2[s][r0 + 8 * q][c], ok2 ? Gi + pl.g2off[q] : G2, ok2);
        }
    }
    {
        const int s = tid >> 6, xp = (tid >> 5) & 1;
        const int I = I0 + s;
        const bool okx = I < nI && pl.qok;
        const long long base = (okx ? I * XP + pl.qoff : 0);
        const bool oy = okx && pl.yok, oz = okx && pl.zok;
        cpa16(&st.ey[s][xp][c], oy ? E4 + base + pl.cy : E4, oy);
        cpa16(&st.ez[s][xp][c], oz ? E4 + base + pl.cz : E4, oz);
        cpa16(&st.fy[s][xp][c], oy ? F4 + base + pl.cy : F4, oy);
        cpa16(&st.fz[s][xp][c], oz ? F4 + base + pl.cz : F4, oz);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Grid: x = block of DX rows X (fastest, so that the blocks running together
// share the G tiles of one (Y, Z) pair in L2), y = pair of mirror tiles.
__global__ void __launch_bounds__(DTH, 1)
    k_triangle_df(double* H, const float4* E4, const float4* F4, const float2* G2, int P,
                  int nX, int nI) {
    extern __shared__ __align__(16) unsigned char df_raw[];
    DfStage* stg = reinterpret_cast<DfStage*>(df_raw);
    const int nb = (P + DT - 1) / DT;
    int pidx = blockIdx.y, Yb = 0;
    while (pidx >= nb - Yb) {
        pidx -= nb - Yb;
        ++Yb;
    }
    const int Zb = Yb + pidx;
    const int Y0 = Yb * DT, Z0 = Zb * DT, X0 = blockIdx.x * DX;
    const int nXp = (nX + 1) / 2, xp0 = X0 / 2;
    const bool diag = Yb == Zb;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // Accumulators of -H for the mirror outputs: [x pair][i][j]
    f2 h1[2][2][2], l1[2][2][2], h2[2][2][2], l2[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) h1[a][i][j] = l1[a][i][j] = h2[a][i][j] = l2[a][i][j] = 0ull;
    const int nsteps = (nI + DS - 1) / DS;
    const DfPlan plan = df_plan(P, nXp, xp0, Y0, Z0);
    if (nsteps > 0) df_load(stg[0], plan, E4, F4, G2, P, nXp, nI, 0);
    for (int k = 0; k < nsteps; ++k) {
        const DfStage& cur = stg[k & 1];
        if (k + 1 < nsteps) {
            df_load(stg[(k + 1) & 1], plan, E4, F4, G2, P, nXp, nI, (k + 1) * DS);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
#pragma unroll
        for (int st = 0; st < DS; ++st) {
            // G^(Y_i, Z_j) and G^(Z_j, Y_i), the same value in both lanes
            f2 g1h[2][2], g1l[2][2], g2h[2][2], g2l[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float2 a = cur.g1[st][ty + 16 * i][tx + 16 * j];
                    const float2 b = cur.g2[st][tx + 16 * j][ty + 16 * i];
                    g1h[i][j] = pk(a.x, a.x);
                    g1l[i][j] = pk(a.y, a.y);
                    g2h[i][j] = pk(b.x, b.x);
                    g2l[i][j] = pk(b.y, b.y);
                }
#pragma unroll
            for (int xp = 0; xp < 2; ++xp) {
                // {h(x), h(x+1)} and {l(x), l(x+1)} as two 64-bit lanes
                ulonglong2 ey[2], fy[2], ez[2], fz[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    ey[i] = reinterpret_cast<const ulonglong2&>(cur.ey[st][xp][ty + 16 * i]);
                    fy[i] = reinterpret_cast<const ulonglong2&>(cur.fy[st][xp][ty + 16 * i]);
                    ez[i] = reinterpret_cast<const ulonglong2&>(cur.ez[st][xp][tx + 16 * i]);
                    fz[i] = reinterpret_cast<const ulonglong2&>(cur.fz[st][xp][tx + 16 * i]);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        f2 th, tl;
                        df_dot2(ey[i].x, ey[i].y, fz[j].x, fz[j].y, ez[j].x, ez[j].y, fy[i].x,
                                fy[i].y, th, tl);
                        const f2 thn = neg2(th);
                        df_acc(h1[xp][i][j], l1[xp][i][j], th, tl, thn, g1h[i][j], g1l[i][j]);
                        df_acc(h2[xp][i][j], l2[xp][i][j], th, tl, thn, g2h[i][j], g2l[i][j]);
                    }
            }
        }
        __syncthreads();   // the buffer is refilled by the next step's load
    }
    // On a diagonal pair both accumulators cover the same tile and count
    // every (Y, Z) twice.
    const double scale = diag ? -0.5 : -1.0;
#pragma unroll
    for (int xp = 0; xp < 2; ++xp)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int Y = Y0 + ty + 16 * i, Z = Z0 + tx + 16 * j;
                if (Y >= P || Z >= P) continue;
                float a0, a1, b0, b1;
                upk(h1[xp][i][j], a0, a1);
                upk(l1[xp][i][j], b0, b1);
                const int x = X0 + 2 * xp;
                if (x < nX) H[((long long)x * P + Y) * P + Z] += scale * ((double)a0 + (double)b0);
                if (x + 1 < nX)
                    H[((long long)(x + 1) * P + Y) * P + Z] += scale * ((double)a1 + (double)b1);
            }
    if (diag) __syncthreads();   // mirror targets overlap other threads' first targets
#pragma unroll
    for (int xp = 0; xp < 2; ++xp)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int Y = Y0 + ty + 16 * i, Z = Z0 + tx + 16 * j;
                if (Y >= P || Z >= P) continue;
                float a0, a1, b0, b1;
                upk(h2[xp][i][j], a0, a1);
                upk(l2[xp][i][j], b0, b1);
                const int x = X0 + 2 * xp;
                if (x < nX) H[((long long)x * P + Z) * P + Y] += scale * ((double)a0 + (double)b0);
                if (x + 1 < nX)
                    H[((long long)(x + 1) * P + Z) * P + Y] += scale * ((double)a1 + (double)b1);
            }
}

// {h, l} = {fl32(d), fl32(d - fl32(d))}.  The float64 form takes four
// float64-pipe operations (1/64 of the float32 rate on GB300: it kept the
// split kernels' float64 pipe 88 % busy), so for 2^-60 <= |d| < 2^60 the
// split is done on the IEEE-754 fields with integer operations: h rounds the
// 53-bit significand to 24 bits (nearest, ties to even); the signed
// remainder, below 2^29 units of 2^(e - 1075), is rounded to float32 and
// given its exponent.  Bit-identical to the float64 form (checked on the host
// over 2e7 values, ties and carries included).  Other values (zero among
// them) take the float64 form out of line, so that the common path carries
// no predicated float64 operations.
__device__ __noinline__ void split1_f64(double d, float& h, float& l) {
    h = __double2float_rn(d);
    l = __double2float_rn(d - (double)h);   // d - h is exact in float64
}

__device__ __forceinline__ bool split1_int(double d, float& h, float& l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 60 || e >= 1023 + 60) return false;
    const unsigned long long m = (b & 0xfffffffffffffULL) | (1ULL << 52);
    unsigned long long q = m >> 29;
    const unsigned long long rem = m & ((1ULL << 29) - 1);
    if (rem > (1ULL << 28) || (rem == (1ULL << 28) && (q & 1ULL))) ++q;
    const long long rs = (long long)m - (long long)(q << 29);   // |rs| <= 2^28
    int eh = e;
    if (q >> 24) {
        q >>= 1;
        ++eh;
    }
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    h = __uint_as_float(sgn | ((unsigned)(eh - 1023 + 127) << 23) | (unsigned)(q & 0x7fffffULL));
    unsigned lb = __float_as_uint(__int2float_rn((int)rs));
    if (rs != 0) lb += (unsigned)(e - 1075) << 23;
    l = rs != 0 ? __uint_as_float(lb ^ sgn) : 0.f;
    return true;
}

__device__ __forceinline__ void split1(double d, float& h, float& l) {
    if (!split1_int(d, h, l)) split1_f64(d, h, l);
}

// One block per output row (I, q) at a time, threads along the P columns
// (no 64-bit division per element).
__global__ void k_split_pairs(const double* E, int nI, int nX, int P, float4* out) {
    const int nXp = (nX + 1) / 2;
    const long long rows = (long long)nI * nXp;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long I = row / nXp;
        const int x = 2 * (int)(row - I * nXp);
        const double* e0 = E + (I * nX + x) * P;
        float4* o = out + row * P;
        const bool two = x + 1 < nX;
        for (int c = threadIdx.x; c < P; c += blockDim.x) {
            const double d0 = e0[c];
            const double d1 = two ? e0[P + c] : 0.0;
            float h0, l0, h1, l1;
            split1(d0, h0, l0);
            split1(d1, h1, l1);
            o[c] = make_float4(h0, h1, l0, l1);
        }
    }
}

// in and out may be the same buffer: element i's float64 value is replaced
// by its float pair in the same eight bytes.
__global__ void k_split_df(const double* in, long long n, float2* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float h, l;
        split1(in[i], h, l);
        out[i] = make_float2(h, l);
    }
}

unsigned grid_for(long long n) {
    return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
}

}  // namespace

cudaError_t split_df_pairs(const double* E, int nI, int nX, int P, float4* out,
                           cudaStream_t s) {
    const long long n = (long long)nI * ((nX + 1) / 2) * P;
    if (n <= 0) return cudaSuccess;
    const long long rows = (long long)nI * ((nX + 1) / 2);
    k_split_pairs<<<(unsigned)std::min<long long>(rows, 152LL * 16), 128, 0, s>>>(E, nI, nX, P,
                                                                               out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t split_df(const double* in, long long n, float2* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_split_df<<<grid_for(n), 256, 0, s>>>(in, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t triangle_df(double* H, const float4* E4, const float4* F4, const float2* G2, int P,
                        int nX, int nI, cudaStream_t s) {
    if (nX <= 0 || nI <= 0) return cudaSuccess;
    const unsigned nb = cdiv(P, DT);
    const int smem = (int)(2 * sizeof(DfStage));
    cudaError_t e = smem_optin((const void*)k_triangle_df, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(cdiv(nX, DX), nb * (nb + 1) / 2);
    k_triangle_df<<<grid, DTH, smem, s>>>(H, E4, F4, G2, P, nX, nI);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace thc
