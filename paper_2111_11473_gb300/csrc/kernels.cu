// Element-wise, reduction and triangle kernels of the residual engine.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "kernels.cuh"

namespace thc {
namespace {

constexpr int NT = 256;

inline unsigned nblocks(long long n) {
    long long b = (n + NT - 1) / NT;
    if (b > 152LL * 64) b = 152LL * 64;   // grid-stride beyond 64 blocks per SM
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
__global__ void k_split(const T* full, int nb, int o, int v, Blocks<T> out) {
    const int n = o + v;
    const long long total = (long long)nb * n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long a = idx / ((long long)n * n);
        int r = (int)(idx / n % n), c = (int)(idx % n);
        T val = full[idx];
        if (r < o && c < o) out.oo[(a * o + r) * o + c] = val;
        else if (r < o) { if (out.ov) out.ov[(a * o + r) * v + (c - o)] = val; }
        else if (c < o) { if (out.vo) out.vo[(a * v + (r - o)) * o + c] = val; }
        else if (out.vv) out.vv[(a * v + (r - o)) * v + (c - o)] = val;
        else if (r >= c) {
            const long long ra = r - o, cb = c - o, vt = (long long)v * (v + 1) / 2;
            out.vvp[a * vt + ra * (ra + 1) / 2 + cb] = val;
        }
    }
}

// Full v x v matrices from their packed lower triangles (row a holds b <= a).
// Tiles below the diagonal copy rows; tiles above it read the mirror tile and
// write it transposed, so every global access runs along a row.
template <typename T>
__global__ void k_unpack_vv(const T* packed, int nb, int v, T* out) {
    __shared__ T tile[32][33];
    const long long vt = (long long)v * (v + 1) / 2;
    const T* src = packed + (long long)blockIdx.z * vt;
    T* dst = out + (long long)blockIdx.z * v * v;
    const int bx = blockIdx.x, by = blockIdx.y;
    // Source tile rows sr0.., columns sc0.. with sr0 >= sc0.
    const int sr0 = 32 * max(bx, by), sc0 = 32 * min(bx, by);
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = sr0 + j, c = sc0 + threadIdx.x;
        T val = T(0);
        if (r < v && c < v)
            val = r >= c ? src[(long long)r * (r + 1) / 2 + c] : src[(long long)c * (c + 1) / 2 + r];
        tile[j][threadIdx.x] = val;
    }
    __syncthreads();
    const int r0 = 32 * by, c0 = 32 * bx;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        if (r < v && c < v) dst[(long long)r * v + c] = by >= bx ? tile[j][threadIdx.x]
                                                                : tile[threadIdx.x][j];
    }
}

template <typename T>
__global__ void k_transpose(const T* in, T* out, int nb, int rows, int cols) {
    __shared__ T tile[32][33];
    const int a = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const T* src = in + (long long)a * rows * cols;
    T* dst = out + (long long)a * rows * cols;
    for (int j = threadIdx.y; j < 32; j += 8) {
        int r = r0 + j, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[j][threadIdx.x] = src[(long long)r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        int c = c0 + j, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(long long)c * rows + r] = tile[threadIdx.x][j];
    }
}

template <typename T>
__global__ void k_convert(const double* in, T* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

template <typename T>
__global__ void k_to_double(const T* in, double* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

template <typename T>
__global__ void k_alg1(const T* Bbar, const T* Btil, const T* oo, const T* vv,
                       T* C1, T* Ccross, int P, int nb) {
    const long long PP = (long long)P * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < PP;
         idx += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(idx / P), Y = (int)(idx % P);
        const T wo = oo[idx], wv = vv[idx];
        T cross = Ccross[idx];
        for (int a = 0; a < nb; ++a) {
            const T bb = Bbar[a * PP + idx], bt = Btil[a * PP + idx];
            C1[((long long)X * nb + a) * P + Y] = wv * bb - wo * bt;
            cross += bb * bt;
        }
        Ccross[idx] = cross;
    }
}

template <typename T>
__global__ void k_diag_reduce(const T* y, const T* M, int R, int P, int nb, T* out,
                              int ldo, int col0) {
    const long long total = (long long)nb * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(idx / P), X = (int)(idx % P);
        const T* m = M + (long long)a * R * P + X;
        T acc = 0;
        for (int r = 0; r < R; ++r) acc += y[(long long)r * P + X] * m[(long long)r * P];
        out[(long long)X * ldo + col0 + a] = acc;
    }
}

template <typename T>
__global__ void k_w_single(const T* TA, int ldta, const T* Tc, const T* E, T* W, int P,
                           int nb) {
    const long long PP = (long long)P * P, total = PP * nb;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(idx / PP);
        const long long e = idx % PP;
        const int Y = (int)(e / P), Z = (int)(e % P);
        T w = -Tc[e] * E[idx];
        if (Y == Z) w += T(2) * TA[(long long)Y * ldta + a];
        W[idx] = w;
    }
}

template <typename T>
__global__ void k_eps_t1(const T* eps, const T* t1, int o, int v, T* out) {
    const long long tot = (long long)o * v;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / o), i = (int)(e % o);
        out[e] = (eps[o + a] - eps[i]) * t1[(long long)i * v + a];
    }
}

template <typename T>
__global__ void k_lincomb(T* out, long long n, double a, const T* x, double b,
                          const T* y, double c, const T* z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T r = T(a) * x[i];
        if (y) r += T(b) * y[i];
        if (z) r += T(c) * z[i];
        out[i] = r;
    }
}

template <typename T>
__global__ void k_hadamard2(T* out, long long n, const T* a, const T* b, const T* c,
                            const T* d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = c ? a[i] * b[i] - c[i] * d[i] : a[i] * b[i];
}

template <typename T>
__global__ void k_hadamard_batched(T* M, const T* z, long long per, int nb) {
    const long long total = per * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        M[i] *= z[i % per];
}

template <typename T>
__global__ void k_kr(const T* A, const T* B, int na, int nbr, int P, T* out) {
    const long long total = (long long)na * nbr * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(idx % P);
        const long long ia = idx / P;
        const int i = (int)(ia / nbr), a = (int)(ia % nbr);
        out[idx] = A[(long long)i * P + X] * B[(long long)a * P + X];
    }
}

template <typename T>
__global__ void k_scale_rows(const T* y, int R, int P, const T* w, int x0, int nx,
                             T* out) {
    const long long per = (long long)R * P, total = per * nx;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx / per);
        const long long e = idx % per;
        const int Y = (int)(e % P);
        out[idx] = y[e] * w[(long long)(x0 + x) * P + Y];
    }
}

// Tile of the float64 triangle kernel: TXB amplitude indices X and a pair of
// TYZ x TYZ (Y, Z) tiles per block.
constexpr int TXB = 4, TYZ = 32;

// Float32 triangle kernel.  A block owns a 32 x 32 x 32 (X, Y, Z) tile of H;
// lane = X, and the 16 warps form a 4 x 4 grid of 8 x 8 (Y, Z) register tiles.
// Per grid point I the block stages E_I[X][Y-tile | Z-tile], F_I likewise and
// G_I[Y-tile][Z-tile] in shared memory through a 3-stage cp.async pipeline.
// Each thread issues 3 FMA-pipe instructions per (I, X, Y, Z); G is read by
// warp-wide broadcast, E and F by conflict-free 128-bit loads (row pad 4).
// Float64 triangle kernel over pairs of mirror (Y, Z) tiles.
// t^XYZ = E^XY F^XZ + E^XZ F^XY is symmetric in (Y, Z), so one t feeds both
// H^XYZ += t G^YZ and H^XZY += t G^ZY: 7 flops per two outputs (two FP64
// FMA-pipe operations per output instead of three).  A block owns 4 X and the
// tiles (Y0, Z0), (Z0, Y0) with Y0 <= Z0; on a diagonal pair (Y0 = Z0) both
// accumulators land on the same tile, count every element twice, and are
// halved and added one after the other.
constexpr int SIST = 2;

struct TriSym64Stage {
    double g1[SIST][TYZ][TYZ + 1];   // G^YZ, rows Y
    double g2[SIST][TYZ][TYZ + 1];   // G^ZY, rows Z
    double ey[SIST][TXB][TYZ], ez[SIST][TXB][TYZ];
    double fy[SIST][TXB][TYZ], fz[SIST][TXB][TYZ];
};

__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(ok ? 8 : 0));
}

// Stage grid points I0 .. I0 + SIST - 1 of the block's tiles (zeros outside).
__device__ __forceinline__ void sym64_load(TriSym64Stage& st, const double* E, const double* F,
                                           const double* G, int P, int nX, int nI, int I0,
                                           int X0, int Y0, int Z0) {
    const long long PP = (long long)P * P, XP = (long long)nX * P;
    const int tid = threadIdx.x;
    for (int e = tid; e < SIST * TYZ * TYZ; e += 256) {
        const int s = e / (TYZ * TYZ), r = (e / TYZ) % TYZ, c = e % TYZ;
        const int I = I0 + s;
        const bool ok1 = I < nI && Y0 + r < P && Z0 + c < P;
        const bool ok2 = I < nI && Z0 + r < P && Y0 + c < P;
        cp_async8(&st.g1[s][r][c], ok1 ? G + I * PP + (long long)(Y0 + r) * P + Z0 + c : G, ok1);
        cp_async8(&st.g2[s][r][c], ok2 ? G + I * PP + (long long)(Z0 + r) * P + Y0 + c : G, ok2);
    }
    for (int e = tid; e < SIST * TXB * TYZ; e += 256) {
        const int s = e / (TXB * TYZ), x = (e / TYZ) % TXB, c = e % TYZ;
        const int I = I0 + s, X = X0 + x;
        const bool okx = I < nI && X < nX;
        const long long base = I * XP + (long long)X * P;
        const bool oy = okx && Y0 + c < P, oz = okx && Z0 + c < P;
        cp_async8(&st.ey[s][x][c], oy ? E + base + Y0 + c : E, oy);
        cp_async8(&st.ez[s][x][c], oz ? E + base + Z0 + c : E, oz);
        cp_async8(&st.fy[s][x][c], oy ? F + base + Y0 + c : F, oy);
        cp_async8(&st.fz[s][x][c], oz ? F + base + Z0 + c : F, oz);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Float64 triangle kernel over pairs of mirror (Y, Z) tiles.
// t^XYZ = E^XY F^XZ + E^XZ F^XY is symmetric in (Y, Z), so one t feeds both
// H^XYZ += t G^YZ and H^XZY += t G^ZY: 7 flops per two outputs (two FP64
// FMA-pipe operations per output instead of three).  A block owns 4 X and the
// tiles (Y0, Z0), (Z0, Y0) with Y0 <= Z0; on a diagonal pair (Y0 = Z0) both
// accumulators land on the same tile, count every element twice, and are
// halved and added one after the other.  Operands of the next pair of grid
// points are staged with cp.async while the current pair is computed.
__global__ void __launch_bounds__(256) k_triangle_sym64(double* H, const double* E,
                                                        const double* F, const double* G,
                                                        int P, int nX, int nI) {
    extern __shared__ __align__(16) unsigned char sym64_raw[];
    TriSym64Stage* stg = reinterpret_cast<TriSym64Stage*>(sym64_raw);
    const int nb = (P + TYZ - 1) / TYZ;
    int pidx = blockIdx.x, Yb = 0;
    while (pidx >= nb - Yb) {
        pidx -= nb - Yb;
        ++Yb;
    }
    const int Zb = Yb + pidx;
    const int Y0 = Yb * TYZ, Z0 = Zb * TYZ, X0 = blockIdx.y * TXB;
    const bool diag = Yb == Zb;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double a1[TXB][2][2], a2[TXB][2][2];
#pragma unroll
    for (int x = 0; x < TXB; ++x)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) a1[x][i][j] = a2[x][i][j] = 0;
    const int nsteps = (nI + SIST - 1) / SIST;
    if (nsteps > 0) sym64_load(stg[0], E, F, G, P, nX, nI, 0, X0, Y0, Z0);
    for (int k = 0; k < nsteps; ++k) {
        const TriSym64Stage& cur = stg[k & 1];
        if (k + 1 < nsteps) {
            sym64_load(stg[(k + 1) & 1], E, F, G, P, nX, nI, (k + 1) * SIST, X0, Y0, Z0);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
#pragma unroll
        for (int st = 0; st < SIST; ++st) {
            double g1[2][2], g2[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    g1[i][j] = cur.g1[st][ty + 16 * i][tx + 16 * j];   // G^(Y_i, Z_j)
                    g2[i][j] = cur.g2[st][tx + 16 * j][ty + 16 * i];   // G^(Z_j, Y_i)
                }
#pragma unroll
            for (int x = 0; x < TXB; ++x) {
                double ey[2], fy[2], ez[2], fz[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    ey[i] = cur.ey[st][x][ty + 16 * i];
                    fy[i] = cur.fy[st][x][ty + 16 * i];
                    ez[i] = cur.ez[st][x][tx + 16 * i];
                    fz[i] = cur.fz[st][x][tx + 16 * i];
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        double t = ey[i] * fz[j];
                        t = fma(ez[j], fy[i], t);
                        a1[x][i][j] = fma(t, g1[i][j], a1[x][i][j]);
                        a2[x][i][j] = fma(t, g2[i][j], a2[x][i][j]);
                    }
            }
        }
        __syncthreads();   // the buffer is refilled two steps later
    }
    const double scale = diag ? 0.5 : 1.0;
#pragma unroll
    for (int x = 0; x < TXB; ++x) {
        const int X = X0 + x;
        if (X >= nX) continue;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int Y = Y0 + ty + 16 * i;
            if (Y >= P) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int Z = Z0 + tx + 16 * j;
                if (Z < P) H[((long long)X * P + Y) * P + Z] += scale * a1[x][i][j];
            }
        }
    }
    if (diag) __syncthreads();   // a2 targets overlap other threads' a1 targets
#pragma unroll
    for (int x = 0; x < TXB; ++x) {
        const int X = X0 + x;
        if (X >= nX) continue;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int Y = Y0 + ty + 16 * i;
            if (Y >= P) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int Z = Z0 + tx + 16 * j;
                if (Z < P) H[((long long)X * P + Z) * P + Y] += scale * a2[x][i][j];
            }
        }
    }
}

constexpr int TT = 32, TROW = 2 * TT + 4, TGROW = TT + 4, TSTAGES = 3;

struct TriStage {
    float e[TT][TROW];
    float f[TT][TROW];
    float g[TT][TGROW];
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = ok ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n));
}

__device__ __forceinline__ void tri_load(TriStage& st, const float* E, const float* F,
                                         const float* G, int I, int P, int nX, int X0, int Y0,
                                         int Z0) {
    const long long PP = (long long)P * P, XP = (long long)nX * P;
    const float* Ei = E + I * XP;
    const float* Fi = F + I * XP;
    const float* Gi = G + I * PP;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = t + 512 * k;
        const int r = e >> 6, c = e & 63;
        const int X = X0 + r;
        const int col = c < TT ? Y0 + c : Z0 + (c - TT);
        const bool ok = X < nX && col < P;
        const long long off = ok ? (long long)X * P + col : 0;
        cp_async4(&st.e[r][c], Ei + off, ok);
        cp_async4(&st.f[r][c], Fi + off, ok);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = t + 512 * k;
        const int r = e >> 5, c = e & 31;
        const bool ok = Y0 + r < P && Z0 + c < P;
        const long long off = ok ? (long long)(Y0 + r) * P + Z0 + c : 0;
        cp_async4(&st.g[r][c], Gi + off, ok);
    }
}

__global__ void __launch_bounds__(512, 1) k_triangle_f32(float* H, const float* E,
                                                         const float* F, const float* G,
                                                         int P, int nX, int nI) {
    extern __shared__ __align__(16) unsigned char tri_smem[];
    TriStage* st = reinterpret_cast<TriStage*>(tri_smem);
    const int Z0 = blockIdx.x * TT, Y0 = blockIdx.y * TT, X0 = blockIdx.z * TT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wy = warp >> 2, wz = warp & 3;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int s = 0; s < TSTAGES - 1; ++s) {
        if (s < nI) tri_load(st[s], E, F, G, s, P, nX, X0, Y0, Z0);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    for (int I = 0; I < nI; ++I) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(TSTAGES - 2));
        __syncthreads();
        const int nxt = I + TSTAGES - 1;
        if (nxt < nI) tri_load(st[nxt % TSTAGES], E, F, G, nxt, P, nX, X0, Y0, Z0);
        asm volatile("cp.async.commit_group;\n" ::);
        const TriStage& c = st[I % TSTAGES];
        float ey[8], fy[8], ez[8], fz[8];
        const float4* er = reinterpret_cast<const float4*>(&c.e[lane][0]);
        const float4* fr = reinterpret_cast<const float4*>(&c.f[lane][0]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float4 a = er[wy * 2 + q], b = fr[wy * 2 + q];
            float4 d = er[8 + wz * 2 + q], h = fr[8 + wz * 2 + q];
            ey[4 * q] = a.x; ey[4 * q + 1] = a.y; ey[4 * q + 2] = a.z; ey[4 * q + 3] = a.w;
            fy[4 * q] = b.x; fy[4 * q + 1] = b.y; fy[4 * q + 2] = b.z; fy[4 * q + 3] = b.w;
            ez[4 * q] = d.x; ez[4 * q + 1] = d.y; ez[4 * q + 2] = d.z; ez[4 * q + 3] = d.w;
            fz[4 * q] = h.x; fz[4 * q + 1] = h.y; fz[4 * q + 2] = h.z; fz[4 * q + 3] = h.w;
        }
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) {
            const float4* gr = reinterpret_cast<const float4*>(&c.g[wy * 8 + yy][wz * 8]);
            const float4 g0 = gr[0], g1 = gr[1];
            const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
            for (int zz = 0; zz < 8; ++zz) {
                float t = ey[yy] * fz[zz];
                t = fmaf(ez[zz], fy[yy], t);
                acc[yy][zz] = fmaf(t, g[zz], acc[yy][zz]);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    const int X = X0 + lane;
    if (X >= nX) return;
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        const int Y = Y0 + wy * 8 + yy;
        if (Y >= P) continue;
        float* h = H + ((long long)X * P + Y) * P;
#pragma unroll
        for (int zz = 0; zz < 8; ++zz) {
            const int Z = Z0 + wz * 8 + zz;
            if (Z < P) h[Z] += acc[yy][zz];
        }
    }
}


__device__ double block_sum(double v) {
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

constexpr int NPART = 512;

template <typename T>
__global__ void k_dot_part(const T* a, const T* b, long long n, double* part) {
    double acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_parts(const double* part, int n, double* out) {
    double acc = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = acc;
}

template <typename T>
__global__ void k_singles_energy(const T* Lov, const T* Mo, const T* t1, int o, int v,
                                 double* part) {
    const int k = blockIdx.x;
    const T* L = Lov + (long long)k * o * v;
    const T* M = Mo + (long long)k * o * o;
    double s = 0, q = 0;
    for (int e = threadIdx.x; e < o * v; e += blockDim.x) s += (double)L[e] * (double)t1[e];
    for (int e = threadIdx.x; e < o * o; e += blockDim.x) {
        int i = e / o, j = e % o;
        q += (double)M[e] * (double)M[j * o + i];
    }
    s = block_sum(s);
    __syncthreads();
    q = block_sum(q);
    if (threadIdx.x == 0) part[k] = 2.0 * s * s - q;
}

__global__ void k_nonfinite(const double* a, long long n, int* flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) atomicOr(flag, 1);
}

template <typename T>
__global__ void k_accumulate(double* acc, const T* part, long long n, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc[i] += scale * (double)part[i];
}

}  // namespace

template <typename T>
cudaError_t split_blocks(const T* full, int nb, int o, int v, Blocks<T> out,
                         cudaStream_t s) {
    long long n = (long long)nb * (o + v) * (o + v);
    k_split<T><<<nblocks(n), NT, 0, s>>>(full, nb, o, v, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t unpack_vv(const T* packed, int nb, int v, T* out, cudaStream_t s) {
    dim3 grid(cdiv(v, 32), cdiv(v, 32), nb);
    k_unpack_vv<T><<<grid, dim3(32, 8), 0, s>>>(packed, nb, v, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t transpose_batched(const T* in, T* out, int nb, int rows, int cols,
                              cudaStream_t s) {
    dim3 grid(cdiv(cols, 32), cdiv(rows, 32), nb);
    k_transpose<T><<<grid, dim3(32, 8), 0, s>>>(in, out, nb, rows, cols);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t convert(const double* in, T* out, long long n, cudaStream_t s) {
    k_convert<T><<<nblocks(n), NT, 0, s>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t to_double(const T* in, double* out, long long n, cudaStream_t s) {
    k_to_double<T><<<nblocks(n), NT, 0, s>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t alg1_combine(const T* Bbar, const T* Btil, const T* oo, const T* vv,
                         T* C1, T* Ccross, int P, int nb, cudaStream_t s) {
    k_alg1<T><<<nblocks((long long)P * P), NT, 0, s>>>(Bbar, Btil, oo, vv, C1, Ccross, P, nb);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t diag_reduce(const T* y, const T* M, int R, int P, int nb, T* out, int ldo,
                        int col0, cudaStream_t s) {
    k_diag_reduce<T><<<nblocks((long long)nb * P), NT, 0, s>>>(y, M, R, P, nb, out, ldo, col0);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t w_single(const T* TA, int ldta, const T* Tc, const T* E, T* W, int P, int nb,
                     cudaStream_t s) {
    k_w_single<T><<<nblocks((long long)nb * P * P), NT, 0, s>>>(TA, ldta, Tc, E, W, P, nb);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t eps_t1(const T* eps, const T* t1, int o, int v, T* out, cudaStream_t s) {
    k_eps_t1<T><<<nblocks((long long)o * v), NT, 0, s>>>(eps, t1, o, v, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t lincomb(T* out, long long n, double a, const T* x, double b, const T* y,
                    double c, const T* z, cudaStream_t s) {
    k_lincomb<T><<<nblocks(n), NT, 0, s>>>(out, n, a, x, b, y, c, z);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hadamard2(T* out, long long n, const T* a, const T* b, const T* c,
                      const T* d, cudaStream_t s) {
    k_hadamard2<T><<<nblocks(n), NT, 0, s>>>(out, n, a, b, c, d);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hadamard_batched(T* M, const T* z, long long per, int nb, cudaStream_t s) {
    k_hadamard_batched<T><<<nblocks(per * nb), NT, 0, s>>>(M, z, per, nb);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t khatri_rao(const T* A, const T* B, int na, int nbr, int P, T* out,
                       cudaStream_t s) {
    k_kr<T><<<nblocks((long long)na * nbr * P), NT, 0, s>>>(A, B, na, nbr, P, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t scale_rows(const T* y, int R, int P, const T* w, int x0, int nx, T* out,
                       cudaStream_t s) {
    k_scale_rows<T><<<nblocks((long long)R * P * nx), NT, 0, s>>>(y, R, P, w, x0, nx, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t triangle(T* H, const T* E, const T* F, const T* G, int P, int nX, int nI,
                     cudaStream_t s) {
    if (nX <= 0 || nI <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        const int smem = (int)(TSTAGES * sizeof(TriStage));
        cudaError_t e = smem_optin((const void*)k_triangle_f32, smem);
        if (e != cudaSuccess) return e;
        dim3 grid(cdiv(P, TT), cdiv(P, TT), cdiv(nX, TT));
        k_triangle_f32<<<grid, 512, smem, s>>>(H, E, F, G, P, nX, nI);
        count_launches(1);
        return cudaGetLastError();
    }
    if constexpr (std::is_same<T, double>::value) {
        const unsigned nb = cdiv(P, TYZ);
        dim3 grid(nb * (nb + 1) / 2, cdiv(nX, TXB));
        const int smem = (int)(2 * sizeof(TriSym64Stage));
        cudaError_t e = smem_optin((const void*)k_triangle_sym64, smem);
        if (e != cudaSuccess) return e;
        k_triangle_sym64<<<grid, 256, smem, s>>>(H, E, F, G, P, nX, nI);
        count_launches(1);
        return cudaGetLastError();
    }
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t dot(const T* a, const T* b, long long n, double* scratch, double* out,
                cudaStream_t s) {
    k_dot_part<T><<<NPART, NT, 0, s>>>(a, b, n, scratch);
    count_launches(1);
    k_sum_parts<<<1, NT, 0, s>>>(scratch, NPART, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t singles_energy(const T* Lov, const T* Mo, const T* t1, int K, int o, int v,
                           double* scratch, double* out, cudaStream_t s) {
    k_singles_energy<T><<<K, NT, 0, s>>>(Lov, Mo, t1, o, v, scratch);
    count_launches(1);
    k_sum_parts<<<1, NT, 0, s>>>(scratch, K, out);
    return cudaGetLastError();
}

cudaError_t any_nonfinite(const double* a, long long n, int* flag, cudaStream_t s) {
    k_nonfinite<<<nblocks(n), NT, 0, s>>>(a, n, flag);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t accumulate(double* acc, const T* part, long long n, double scale,
                       cudaStream_t s) {
    k_accumulate<T><<<nblocks(n), NT, 0, s>>>(acc, part, n, scale);
    count_launches(1);
    return cudaGetLastError();
}

#define THC_INSTANTIATE(T)                                                              \
    template cudaError_t split_blocks<T>(const T*, int, int, int, Blocks<T>, cudaStream_t); \
    template cudaError_t unpack_vv<T>(const T*, int, int, T*, cudaStream_t);            \
    template cudaError_t transpose_batched<T>(const T*, T*, int, int, int, cudaStream_t); \
    template cudaError_t convert<T>(const double*, T*, long long, cudaStream_t);        \
    template cudaError_t to_double<T>(const T*, double*, long long, cudaStream_t);      \
    template cudaError_t alg1_combine<T>(const T*, const T*, const T*, const T*, T*, T*, \
                                         int, int, cudaStream_t);                       \
    template cudaError_t diag_reduce<T>(const T*, const T*, int, int, int, T*, int, int, \
                                        cudaStream_t);                                  \
    template cudaError_t w_single<T>(const T*, int, const T*, const T*, T*, int, int,  \
                                     cudaStream_t);                                     \
    template cudaError_t eps_t1<T>(const T*, const T*, int, int, T*, cudaStream_t);     \
    template cudaError_t lincomb<T>(T*, long long, double, const T*, double, const T*, \
                                    double, const T*, cudaStream_t);                    \
    template cudaError_t hadamard2<T>(T*, long long, const T*, const T*, const T*,     \
                                      const T*, cudaStream_t);                          \
    template cudaError_t hadamard_batched<T>(T*, const T*, long long, int, cudaStream_t); \
    template cudaError_t khatri_rao<T>(const T*, const T*, int, int, int, T*, cudaStream_t); \
    template cudaError_t scale_rows<T>(const T*, int, int, const T*, int, int, T*,     \
                                       cudaStream_t);                                   \
    template cudaError_t triangle<T>(T*, const T*, const T*, const T*, int, int, int,  \
                                     cudaStream_t);                                     \
    template cudaError_t dot<T>(const T*, const T*, long long, double*, double*,       \
                                cudaStream_t);                                          \
    template cudaError_t singles_energy<T>(const T*, const T*, const T*, int, int, int, \
                                           double*, double*, cudaStream_t);             \
    template cudaError_t accumulate<T>(double*, const T*, long long, double, cudaStream_t);

THC_INSTANTIATE(double)
THC_INSTANTIATE(float)

}  // namespace thc
