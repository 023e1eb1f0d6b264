// Eigenvalue-weighted CP-ALS of the rank-reduced projectors (Eqs. 15-16,
// App. I): U_ia^P ~ sum_W y_i^W y_a^W tau^PW, minimising
//   f = sum_P eps_P^2 sum_ia (U_ia^P - sum_W y_i^W y_a^W tau^PW)^2
// by alternating least squares over y_o, y_v and tau, in float64 on the
// device.  The right-hand sides are products with the weighted factors
// (the MTTKRP of App. I's Eq. 46 as one GEMM plus a reduction over the
// other orbital index); the W x W normal equations (Eqs. 44-45) are solved
// by Cholesky factorisation instead of App. I's preconditioned CG.
#include <cusolverDn.h>

#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

namespace thc {

void set_thread_error(const std::string& msg);

namespace {

unsigned nblk(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152 * 16); }

// te[P][X] = eps_P^2 tau[P][X]
__global__ void k_weight_rows(const double* tau, const double* eps, int N, int W, double* te) {
    const long long tot = (long long)N * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const double w = eps[e / W];
        te[e] = w * w * tau[e];
    }
}

// occ = 1: R[i][X] = sum_a M[(i,a)][X] yv[a][X];  occ = 0: R[a][X] = sum_i M[(i,a)][X] yo[i][X]
__global__ void k_reduce_other(const double* M, const double* f, int o, int v, int W, int occ,
                               double* R) {
    const int rows = occ ? o : v, other = occ ? v : o;
    const long long tot = (long long)rows * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / W), X = (int)(e % W);
        double s = 0;
        for (int q = 0; q < other; ++q) {
            const long long row = occ ? (long long)r * v + q : (long long)q * v + r;
            s += M[row * W + X] * f[(long long)q * W + X];
        }
        R[e] = s;
    }
}

// KR[(i,a)][X] = yo[i][X] yv[a][X]
__global__ void k_khatri_rao(const double* yo, const double* yv, int o, int v, int W, double* KR) {
    const long long tot = (long long)o * v * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const long long row = e / W;
        const int X = (int)(e % W), i = (int)(row / v), a = (int)(row % v);
        KR[e] = yo[(long long)i * W + X] * yv[(long long)a * W + X];
    }
}

__global__ void k_mul(double* a, const double* b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        a[e] *= b[e];
}

// part[block] = sum over its elements of (eps_P (U - rec))^2, U, rec: (ov) x N
__global__ void k_wsq(const double* U, const double* rec, const double* eps, long long rows,
                      int N, double* part) {
    __shared__ double red[32];
    double s = 0;
    const long long tot = rows * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const double d = eps[e % N] * (U[e] - rec[e]);
        s += d * d;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = s;
    __syncthreads();
    if (w == 0) {
        s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) part[blockIdx.x] = s;
    }
}

struct Dev {
    double* p = nullptr;
    ~Dev() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, n * sizeof(double)); }
};

// C (M x N) = alpha A B + beta C, row-major views.
cudaError_t gemm(cudaStream_t st, int M, int N, int K, View<double> A, View<double> B, double* C,
                 long long ldc, double alpha, double beta, double* ws, size_t ws_elems) {
    Gemm<double> g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.B = B; g.C = C; g.ldc = ldc;
    g.alpha = alpha; g.beta = beta;
    g.ws = ws; g.ws_elems = ws_elems;
    return gemm_simt(g, st);
}

View<double> rmv(const double* p, long long ld) { return View<double>{p, ld, 1}; }
View<double> trv(const double* p, long long ld) { return View<double>{p, 1, ld}; }

struct Als {
    int o, v, N, W;
    long long ov;
    cudaStream_t st;
    cusolverDnHandle_t h = nullptr;
    Dev S, S2, M, KR, R, te, rec, part, ws, work, info;
    int lwork = 0;
    std::string err;

    ~Als() { if (h) cusolverDnDestroy(h); }

    cudaError_t init() {
        cudaError_t e;
        if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return cudaErrorUnknown;
        cusolverDnSetStream(h, st);
        const long long mx = std::max<long long>(std::max<long long>(o, v), N);
        if ((e = S.alloc((size_t)W * W)) || (e = S2.alloc((size_t)W * W)) ||
            (e = M.alloc((size_t)ov * W)) || (e = KR.alloc((size_t)ov * W)) ||
            (e = R.alloc((size_t)mx * W)) || (e = te.alloc((size_t)N * W)) ||
            (e = rec.alloc((size_t)ov * N)) || (e = part.alloc(152 * 16)) ||
            (e = ws.alloc(1 << 22)))
            return e;
        if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_UPPER, W, S.p, W, &lwork) !=
            CUSOLVER_STATUS_SUCCESS)
            return cudaErrorUnknown;
        if ((e = work.alloc((size_t)std::max(lwork, 1))) || (e = info.alloc(1))) return e;
        return cudaSuccess;
    }

    // S = (Aᵀ A) o (Bᵀ B) for row-major A (na x W), B (nb x W)
    cudaError_t gram2(const double* A, int na, const double* B, int nb) {
        cudaError_t e;
        if ((e = gemm(st, W, W, na, trv(A, W), rmv(A, W), S.p, W, 1, 0, ws.p, 1 << 22))) return e;
        if ((e = gemm(st, W, W, nb, trv(B, W), rmv(B, W), S2.p, W, 1, 0, ws.p, 1 << 22))) return e;
        k_mul<<<nblk((long long)W * W), 256, 0, st>>>(S.p, S2.p, (long long)W * W);
        count_launches(1);
        return cudaGetLastError();
    }

    // out (rows x W, row-major) = R S^-1 by Cholesky of the symmetric S.
    cudaError_t solve(int rows, double* out) {
        cudaError_t e;
        int hinfo = 0;
        if ((e = cudaMemcpyAsync(S2.p, S.p, sizeof(double) * W * W, cudaMemcpyDeviceToDevice, st)))
            return e;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, W, S.p, W, work.p, lwork, (int*)info.p) !=
                CUSOLVER_STATUS_SUCCESS)
                return cudaErrorUnknown;
            if ((e = cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st)))
                return e;
            if (hinfo == 0) break;
            // Numerically singular: retry once with a ridge of 1e-12 of the largest diagonal.
            std::vector<double> hs((size_t)W * W);
            if ((e = cudaMemcpy(hs.data(), S2.p, sizeof(double) * W * W, cudaMemcpyDeviceToHost)))
                return e;
            double dmax = 0;
            for (int k = 0; k < W; ++k) dmax = std::max(dmax, std::fabs(hs[(size_t)k * W + k]));
            for (int k = 0; k < W; ++k) hs[(size_t)k * W + k] += 1e-12 * dmax;
            if ((e = cudaMemcpy(S.p, hs.data(), sizeof(double) * W * W, cudaMemcpyHostToDevice)))
                return e;
        }
        if (hinfo != 0) {
            err = "cp_als: normal equations are singular";
            return cudaErrorInvalidValue;
        }
        if ((e = cudaMemcpyAsync(out, R.p, sizeof(double) * rows * W, cudaMemcpyDeviceToDevice, st)))
            return e;
        // out viewed column-major is W x rows = R^T; S symmetric: S X = R^T.
        if (cusolverDnDpotrs(h, CUBLAS_FILL_MODE_UPPER, W, rows, S.p, W, out, W, (int*)info.p) !=
            CUSOLVER_STATUS_SUCCESS)
            return cudaErrorUnknown;
        return cudaGetLastError();
    }

    cudaError_t objective(const double* U, const double* eps, const double* yo, const double* yv,
                          const double* tau, double* f) {
        cudaError_t e;
        k_khatri_rao<<<nblk(ov * W), 256, 0, st>>>(yo, yv, o, v, W, KR.p);
        count_launches(1);
        if ((e = cudaGetLastError())) return e;
        if ((e = gemm(st, (int)ov, N, W, rmv(KR.p, W), trv(tau, W), rec.p, N, 1, 0, ws.p, 1 << 22)))
            return e;
        const unsigned nb = nblk(ov * N);
        k_wsq<<<nb, 256, 0, st>>>(U, rec.p, eps, ov, N, part.p);
        count_launches(1);
        if ((e = cudaGetLastError())) return e;
        std::vector<double> hp(nb);
        if ((e = cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return e;
        double s = 0;
        for (double x : hp) s += x;
        *f = s;
        return cudaSuccess;
    }

    cudaError_t sweep(const double* U, const double* eps, double* yo, double* yv, double* tau) {
        cudaError_t e;
        // y_o and y_v share M = U diag(eps^2) tau (tau is fixed in both updates)
        k_weight_rows<<<nblk((long long)N * W), 256, 0, st>>>(tau, eps, N, W, te.p);
        count_launches(1);
        if ((e = cudaGetLastError())) return e;
        if ((e = gemm(st, (int)ov, W, N, rmv(U, N), rmv(te.p, W), M.p, W, 1, 0, ws.p, 1 << 22)))
            return e;
        // y_o: S = (y_v^T y_v) o (tau^T E tau)
        if ((e = gemm(st, W, W, N, trv(tau, W), rmv(te.p, W), S2.p, W, 1, 0, ws.p, 1 << 22)))
            return e;
        if ((e = gemm(st, W, W, v, trv(yv, W), rmv(yv, W), S.p, W, 1, 0, ws.p, 1 << 22))) return e;
        k_mul<<<nblk((long long)W * W), 256, 0, st>>>(S.p, S2.p, (long long)W * W);
        k_reduce_other<<<nblk((long long)o * W), 256, 0, st>>>(M.p, yv, o, v, W, 1, R.p);
        count_launches(2);
        if ((e = cudaGetLastError())) return e;
        if ((e = solve(o, yo))) return e;
        // y_v: S = (y_o^T y_o) o (tau^T E tau)
        if ((e = gemm(st, W, W, N, trv(tau, W), rmv(te.p, W), S2.p, W, 1, 0, ws.p, 1 << 22)))
            return e;
        if ((e = gemm(st, W, W, o, trv(yo, W), rmv(yo, W), S.p, W, 1, 0, ws.p, 1 << 22))) return e;
        k_mul<<<nblk((long long)W * W), 256, 0, st>>>(S.p, S2.p, (long long)W * W);
        k_reduce_other<<<nblk((long long)v * W), 256, 0, st>>>(M.p, yo, o, v, W, 0, R.p);
        count_launches(2);
        if ((e = cudaGetLastError())) return e;
        if ((e = solve(v, yv))) return e;
        // tau: S = (y_o^T y_o) o (y_v^T y_v), R = U^T KR(y_o, y_v)
        if ((e = gram2(yo, o, yv, v))) return e;
        k_khatri_rao<<<nblk(ov * W), 256, 0, st>>>(yo, yv, o, v, W, KR.p);
        count_launches(1);
        if ((e = cudaGetLastError())) return e;
        if ((e = gemm(st, N, W, (int)ov, trv(U, N), rmv(KR.p, W), R.p, W, 1, 0, ws.p, 1 << 22)))
            return e;
        return solve(N, tau);
    }
};

}  // namespace
}  // namespace thc

extern "C" thc_status thc_cp_als(int n_occ, int n_vir, int n_rr, int rank, const double* U,
                                 const double* eps, double* y_o, double* y_v, double* tau,
                                 int iters, double* objective, void* stream) {
    using namespace thc;
    if (n_occ <= 0 || n_vir <= 0 || n_rr <= 0 || rank <= 0 || iters < 0 || !U || !eps || !y_o ||
        !y_v || !tau) {
        set_thread_error("thc_cp_als: non-positive size or NULL pointer");
        return THC_ERR_ARG;
    }
    Als a;
    a.o = n_occ; a.v = n_vir; a.N = n_rr; a.W = rank;
    a.ov = (long long)n_occ * n_vir;
    a.st = (cudaStream_t)stream;
    cudaError_t e = a.init();
    // Device copies of the inputs and of the factors (updated in place).
    Dev dU, de, dyo, dyv, dt;
    const size_t nU = (size_t)a.ov * n_rr;
    const size_t no = (size_t)n_occ * rank, nv = (size_t)n_vir * rank, nt = (size_t)n_rr * rank;
    if (!e) e = dU.alloc(nU);
    if (!e) e = de.alloc(n_rr);
    if (!e) e = dyo.alloc(no);
    if (!e) e = dyv.alloc(nv);
    if (!e) e = dt.alloc(nt);
    if (!e) e = cudaMemcpyAsync(dU.p, U, sizeof(double) * nU, cudaMemcpyDefault, a.st);
    if (!e) e = cudaMemcpyAsync(de.p, eps, sizeof(double) * n_rr, cudaMemcpyDefault, a.st);
    if (!e) e = cudaMemcpyAsync(dyo.p, y_o, sizeof(double) * no, cudaMemcpyDefault, a.st);
    if (!e) e = cudaMemcpyAsync(dyv.p, y_v, sizeof(double) * nv, cudaMemcpyDefault, a.st);
    if (!e) e = cudaMemcpyAsync(dt.p, tau, sizeof(double) * nt, cudaMemcpyDefault, a.st);
    for (int it = 0; it < iters && !e; ++it) {
        e = a.sweep(dU.p, de.p, dyo.p, dyv.p, dt.p);
        if (!e && objective) {
            double f = 0;
            e = a.objective(dU.p, de.p, dyo.p, dyv.p, dt.p, &f);
            if (!e) objective[it] = f;
        }
    }
    if (!e) e = cudaMemcpyAsync(y_o, dyo.p, sizeof(double) * no, cudaMemcpyDefault, a.st);
    if (!e) e = cudaMemcpyAsync(y_v, dyv.p, sizeof(double) * nv, cudaMemcpyDefault, a.st);
    if (!e) e = cudaMemcpyAsync(tau, dt.p, sizeof(double) * nt, cudaMemcpyDefault, a.st);
    if (!e) e = cudaStreamSynchronize(a.st);
    if (e) {
        set_thread_error(a.err.empty() ? std::string("thc_cp_als: ") + cudaGetErrorString(e)
                                       : "thc_cp_als: " + a.err);
        return a.err.empty() ? THC_ERR_CUDA : THC_ERR_NUMERIC;
    }
    return THC_OK;
}
