// Element-wise, reduction and triangle kernels of the residual engine.
#pragma once

#include "common.cuh"

namespace thc {

// Blocks of the Cholesky vectors of one slab (or of h, with nb = 1).
template <typename T>
struct Blocks {
    T* oo = nullptr;  // nb x o x o
    T* ov = nullptr;  // nb x o x v
    T* vo = nullptr;  // nb x v x o
    T* vv = nullptr;  // nb x v x v
    T* vvp = nullptr; // nb x v(v+1)/2: lower triangle of the vv block, row a
                      // holding b = 0..a (written when vv is null)
};

template <typename T>
cudaError_t split_blocks(const T* full, int nb, int o, int v, Blocks<T> out,
                         cudaStream_t s);
// out[k] (v x v) = the symmetric matrix whose lower triangle is packed[k].
template <typename T>
cudaError_t unpack_vv(const T* packed, int nb, int v, T* out, cudaStream_t s);
template <typename T>
cudaError_t transpose_batched(const T* in, T* out, int nb, int rows, int cols,
                              cudaStream_t s);
template <typename T>
cudaError_t convert(const double* in, T* out, long long n, cudaStream_t s);
template <typename T>
cudaError_t to_double(const T* in, double* out, long long n, cudaStream_t s);

// C1[X][a][Y] = v[X,Y] Bbar[a][X][Y] - o[X,Y] Btil[a][X][Y];
// Ccross[X][Y] += sum_a Bbar[a][X][Y] Btil[a][X][Y].
template <typename T>
cudaError_t alg1_combine(const T* Bbar, const T* Btil, const T* oo, const T* vv,
                         T* C1, T* Ccross, int P, int nb, cudaStream_t s);

// out[X * ldo + col0 + a] = sum_r y[r][X] M[a][r][X],  a < nb, r < R.
template <typename T>
cudaError_t diag_reduce(const T* y, const T* M, int R, int P, int nb, T* out,
                        int ldo, int col0, cudaStream_t s);

// W[a][Y][Z] = 2 d(Y,Z) TA[Y * ldta + a] - T[Y][Z] E[a][Y][Z].
template <typename T>
cudaError_t w_single(const T* TA, int ldta, const T* Tc, const T* E, T* W, int P,
                     int nb, cudaStream_t s);

// out[a][i] = (eps[o + a] - eps[i]) t1[i][a]   (v x o; the orbital-energy part
// of the T1-dressed diagonal Fock matrix, block (a, i)).
template <typename T>
cudaError_t eps_t1(const T* eps, const T* t1, int o, int v, T* out, cudaStream_t s);

// out = a*x + b*y + c*z element-wise (z may be null).
template <typename T>
cudaError_t lincomb(T* out, long long n, double a, const T* x, double b,
                    const T* y, double c, const T* z, cudaStream_t s);

// out = a o b - c o d (Hadamard), n elements; c = d = null gives a o b.
template <typename T>
cudaError_t hadamard2(T* out, long long n, const T* a, const T* b, const T* c,
                      const T* d, cudaStream_t s);

// M[k][i][j] *= z[i][j] for nb G x G matrices.
template <typename T>
cudaError_t hadamard_batched(T* M, const T* z, long long per, int nb,
                             cudaStream_t s);

// KR[(i,a)][X] = A[i][X] B[a][X].
template <typename T>
cudaError_t khatri_rao(const T* A, const T* B, int na, int nbr, int P, T* out,
                       cudaStream_t s);

// Yv[x][i][Y] = y[i][Y] w[(x0+x)][Y]   (scaled copies of a factor matrix).
template <typename T>
cudaError_t scale_rows(const T* y, int R, int P, const T* w, int x0, int nx,
                       T* out, cudaStream_t s);

// Alg. 6 line 11: H[X][Y][Z] += sum_I (E_I^XY F_I^XZ + E_I^XZ F_I^XY) G_I^YZ
// for a block of nX rows X (X < nX <= P, Y, Z < P): H is nX x P x P, E and F
// are nI x nX x P, G is nI x P x P.  Float64: mirror (Y, Z) tiles on the
// FP64 pipe; float32: 32^3 tiles through cp.async (the mixed path takes
// triangle_pair when P is a multiple of 4).
template <typename T>
cudaError_t triangle(T* H, const T* E, const T* F, const T* G, int P, int nX, int nI,
                     cudaStream_t s);

// Float64-accurate triangle on the FP32 pipe (float pairs, error-free
// transformations; triangle_df.cu).  E4, F4: nI x ceil(nX/2) x P float4
// {h(x), h(x+1), l(x), l(x+1)} of E^{xY} for the row pairs x = 2q, 2q + 1
// (split_df_pairs); G2: nI x P x P float2 {h, l} (split_df); H: nX x P x P
// float64, accumulated into.
cudaError_t split_df_pairs(const double* E, int nI, int nX, int P, float4* out,
                           cudaStream_t s);
// out[i] = {fl32(in[i]), fl32(in[i] - fl32(in[i]))}; out may alias in.
cudaError_t split_df(const double* in, long long n, float2* out, cudaStream_t s);
cudaError_t triangle_df(double* H, const float4* E4, const float4* F4, const float2* G2, int P,
                        int nX, int nI, cudaStream_t s);

// Float32 triangle over X pairs in packed lanes (triangle_pair.cu), for P a
// multiple of 4 and at most kPairMaxP.  E2, F2: nI x ceil(nX/2) x P float2
// {E^{2q,Y}, E^{2q+1,Y}} (16-byte aligned); G: nI x P x P; H: nX x P x P,
// accumulated into.  err (device int) receives 1 if a bounded wait expired.
constexpr int kPairMaxP = 28000;
bool triangle_pair_ok(int P);
cudaError_t triangle_pair(float* H, const float2* E2, const float2* F2, const float* G, int P,
                          int nX, int nI, cudaStream_t s, int* err);
// In place: for each of nslab slabs at A + b stride (stride >= nX rounded up
// to even, times P), rows 2q, 2q + 1 of P floats become the interleaved
// pairs of triangle_pair's layout (0 in the second lane of an odd last row).
cudaError_t pair_rows(float* A, long long nslab, long long stride, int nX, int P,
                      cudaStream_t s);

// Deterministic float64 sums.
// out[0] = sum_i a[i] b[i]
template <typename T>
cudaError_t dot(const T* a, const T* b, long long n, double* scratch,
                double* out, cudaStream_t s);
// out[0] = sum_k [2 (sum_ia L_k,ia t_ia)^2 - sum_ij M_k,ij M_k,ji], M_k = L_k t^T
template <typename T>
cudaError_t singles_energy(const T* Lov, const T* Mo, const T* t1, int K, int o,
                           int v, double* scratch, double* out, cudaStream_t s);

// flag[0] = 1 if any of n values is not finite.
cudaError_t any_nonfinite(const double* a, long long n, int* flag, cudaStream_t s);

// sigma_d += (double) sigma_r element-wise (accumulation of float partials).
template <typename T>
cudaError_t accumulate(double* acc, const T* part, long long n, double scale,
                       cudaStream_t s);

}  // namespace thc
