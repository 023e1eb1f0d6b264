// Jacobi + DIIS solver of the projected THC-RR-CCSD amplitude equations.
//
// The paper states only that the residual is converged to 1e-8 (Fig. 3); the
// update is the orbital-energy Jacobi step in the orthonormal basis of Eq. 22
// (the working variable T^PQ the paper recommends) with Pulay DIIS, all in
// float64 on the device.  The only host arithmetic is the (m+1) x (m+1) DIIS
// system.
#include <cusolverDn.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "solver.cuh"

namespace thc {

namespace {

using View64 = View<double>;
View64 rm64(const double* p, long long ld) { return View64{p, ld, 1}; }
View64 tr64(const double* p, long long ld) { return View64{p, 1, ld}; }

__global__ void k_scale_diag(const double* y, const double* eps, int R, int P, double* out) {
    const long long total = (long long)R * P;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = y[i] * eps[i / P];
}

__global__ void k_metric(const double* oo, const double* vv, const double* oe,
                         const double* ve, double* S, double* F, long long nn) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
         i += (long long)gridDim.x * blockDim.x) {
        S[i] = oo[i] * vv[i];
        F[i] = oo[i] * ve[i] - oe[i] * vv[i];
    }
}

// X[i][k] = V[(k0 + k) * P + i] / sqrt(s[k0 + k])   (cuSOLVER returns V column-major)
__global__ void k_half_inverse(const double* V, const double* s, int P, int k0, int r,
                               double* X) {
    const long long total = (long long)P * r;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / r), k = (int)(idx % r);
        X[idx] = V[(long long)(k0 + k) * P + i] / sqrt(s[k0 + k]);
    }
}

// row-major W[i][k] from column-major eigenvectors
__global__ void k_colmajor_to_rowmajor(const double* V, int r, double* W) {
    const long long total = (long long)r * r;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / r), k = (int)(idx % r);
        W[idx] = V[(long long)k * r + i];
    }
}

__global__ void k_symmetrize(double* A, int n) {
    const long long total = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        if (i < j) {
            const double m = 0.5 * (A[idx] + A[(long long)j * n + i]);
            A[idx] = m;
            A[(long long)j * n + i] = m;
        }
    }
}

// step = [-sigma1 / (eps_a - eps_i) | -sigma_q / (e_P + e_Q)];  xnew = x + step
__global__ void k_jacobi(const double* sig1, const double* sq, const double* eps,
                         const double* e, int o, int v, int r, const double* x, double* step,
                         double* xnew) {
    const long long ov = (long long)o * v, total = ov + (long long)r * r;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        double s;
        if (idx < ov) {
            const int i = (int)(idx / v), a = (int)(idx % v);
            s = -sig1[idx] / (eps[o + a] - eps[i]);
        } else {
            const long long q = idx - ov;
            const int p = (int)(q / r), qq = (int)(q % r);
            s = -sq[q] / (e[p] + e[qq]);
        }
        step[idx] = s;
        xnew[idx] = x[idx] + s;
    }
}

__global__ void k_combine(const double* hx, const double* c, int m, long long len,
                          double* out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
         idx += (long long)gridDim.x * blockDim.x) {
        double s = 0;
        for (int k = 0; k < m; ++k) s += c[k] * hx[(long long)k * len + idx];
        out[idx] = s;
    }
}

__device__ double block_sum64(double v) {
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// out[k] = <a_k, b> for m vectors a_k (stride len), one block per k.
__global__ void k_multidot(const double* A, const double* b, long long len, double* out) {
    const double* a = A + (long long)blockIdx.x * len;
    double s = 0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) s += a[i] * b[i];
    s = block_sum64(s);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

unsigned nb(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152 * 32); }

// out = a + b (n elements)
__global__ void k_add(const double* a, const double* b, long long n, double* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// out = a - b
__global__ void k_sub(const double* a, const double* b, long long n, double* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// out[k] = src[idx[k]]
__global__ void k_gather64(const double* src, const long long* idx, long long n, double* out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = src[idx[k]];
}

// t[k] = (Tstar[idx[k]] - Tk[k]) / s[k]
__global__ void k_targets(const double* Tstar, const long long* idx, const double* Tk,
                          const double* sk, long long n, float* t) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        t[k] = (float)((Tstar[idx[k]] - Tk[k]) / sk[k]);
}

__global__ void k_fill64(double* p, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Solve the bordered DIIS system; returns false if it is singular.
bool diis_coefficients(const std::vector<double>& Bm, int m, std::vector<double>& c) {
    const int N = m + 1;
    std::vector<double> A((size_t)N * N, 0.0), rhs(N, 0.0);
    double scale = 0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(Bm[(size_t)i * m + i]));
    if (scale <= 0) return false;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[(size_t)i * N + j] = Bm[(size_t)i * m + j] / scale;
    for (int i = 0; i < m; ++i) A[(size_t)i * N + m] = A[(size_t)m * N + i] = -1.0;
    rhs[m] = -1.0;
    // Gaussian elimination with partial pivoting.
    for (int k = 0; k < N; ++k) {
        int p = k;
        for (int i = k + 1; i < N; ++i)
            if (std::fabs(A[(size_t)i * N + k]) > std::fabs(A[(size_t)p * N + k])) p = i;
        if (std::fabs(A[(size_t)p * N + k]) < 1e-300) return false;
        if (p != k) {
            for (int j = 0; j < N; ++j) std::swap(A[(size_t)k * N + j], A[(size_t)p * N + j]);
            std::swap(rhs[k], rhs[p]);
        }
        for (int i = k + 1; i < N; ++i) {
            const double f = A[(size_t)i * N + k] / A[(size_t)k * N + k];
            for (int j = k; j < N; ++j) A[(size_t)i * N + j] -= f * A[(size_t)k * N + j];
            rhs[i] -= f * rhs[k];
        }
    }
    std::vector<double> sol(N);
    for (int i = N - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int j = i + 1; j < N; ++j) s -= A[(size_t)i * N + j] * sol[j];
        sol[i] = s / A[(size_t)i * N + i];
    }
    c.assign(sol.begin(), sol.begin() + m);
    for (double ci : c)
        if (!std::isfinite(ci)) return false;
    return true;
}

struct Cusolver {
    cusolverDnHandle_t h = nullptr;
    ~Cusolver() { if (h) cusolverDnDestroy(h); }
};

Err syevd(cudaStream_t st, double* A, int N, double* w) {
    Cusolver cs;
    if (cusolverDnCreate(&cs.h) != CUSOLVER_STATUS_SUCCESS)
        return Err{THC_ERR_CUDA, "cusolverDnCreate failed"};
    cusolverDnSetStream(cs.h, st);
    int lwork = 0;
    if (cusolverDnDsyevd_bufferSize(cs.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, N, A,
                                    N, w, &lwork) != CUSOLVER_STATUS_SUCCESS)
        return Err{THC_ERR_CUDA, "syevd buffer size failed"};
    DBuf<double> work;
    DBuf<int> info;
    THC_TRY(work.alloc((size_t)std::max(lwork, 1)));
    THC_TRY(info.alloc(1));
    if (cusolverDnDsyevd(cs.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, N, A, N, w,
                         work.p, lwork, info.p) != CUSOLVER_STATUS_SUCCESS)
        return Err{THC_ERR_CUDA, "syevd failed"};
    int hinfo = 0;
    THC_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    THC_CUDA(cudaStreamSynchronize(st));
    if (hinfo != 0) return Err{THC_ERR_NUMERIC, "metric eigensolver did not converge"};
    return Err{};
}

}  // namespace

Err Solver::mm(cudaStream_t st, int M, int N, int K, View<double> A, View<double> Bv,
               double* Cp, long long ldc, double alpha, double beta) {
    Gemm<double> g;
    g.M = M; g.N = N; g.K = K; g.A = A; g.B = Bv; g.C = Cp; g.ldc = ldc;
    g.alpha = alpha; g.beta = beta;
    g.ws = ws.p; g.ws_elems = ws.n;
    THC_CUDA(gemm_simt(g, st));
    return Err{};
}

template <typename T>
Err Solver::setup(Engine<T>& eng, double cutoff) {
    cudaStream_t st = eng.st;
    P = eng.P; o = eng.o; v = eng.v;
    const int n = o + v;
    const long long PP = (long long)P * P;
    THC_TRY(ws.alloc((size_t)std::max<long long>(4 * PP, 1 << 20)));
    THC_TRY(epsd.alloc(n));
    THC_CUDA(cudaMemcpyAsync(epsd.p, eng.eps_h.data(), sizeof(double) * n,
                             cudaMemcpyHostToDevice, st));
    DBuf<double> yd, yo_e, yv_e, oo, vv, oe, ve, F, Wm, sv;
    THC_TRY(yd.alloc((size_t)n * P));
    if constexpr (std::is_same<T, double>::value) {
        THC_CUDA(cudaMemcpyAsync(yd.p, eng.y.p, sizeof(double) * n * P, cudaMemcpyDeviceToDevice, st));
    } else {
        THC_CUDA(to_double(eng.y.p, yd.p, (long long)n * P, st));
    }
    const double* yo = yd.p;
    const double* yv = yd.p + (long long)o * P;
    THC_TRY(yo_e.alloc((size_t)o * P));
    THC_TRY(yv_e.alloc((size_t)v * P));
    k_scale_diag<<<nb((long long)o * P), 256, 0, st>>>(yo, epsd.p, o, P, yo_e.p);
    count_launches(1);
    k_scale_diag<<<nb((long long)v * P), 256, 0, st>>>(yv, epsd.p + o, v, P, yv_e.p);
    THC_CUDA(cudaGetLastError());
    for (DBuf<double>* b : {&oo, &vv, &oe, &ve, &F}) THC_TRY(b->alloc(PP));
    THC_TRY(Sd.alloc(PP));
    THC_TRY(mm(st, P, P, o, tr64(yo, P), rm64(yo, P), oo.p, P, 1, 0));
    THC_TRY(mm(st, P, P, v, tr64(yv, P), rm64(yv, P), vv.p, P, 1, 0));
    THC_TRY(mm(st, P, P, o, tr64(yo, P), rm64(yo_e.p, P), oe.p, P, 1, 0));
    THC_TRY(mm(st, P, P, v, tr64(yv, P), rm64(yv_e.p, P), ve.p, P, 1, 0));
    k_metric<<<nb(PP), 256, 0, st>>>(oo.p, vv.p, oe.p, ve.p, Sd.p, F.p, PP);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    k_symmetrize<<<nb(PP), 256, 0, st>>>(F.p, P);
    count_launches(1);
    // S = V diag(s) V^T
    THC_TRY(Wm.alloc(PP));
    THC_TRY(sv.alloc(P));
    THC_CUDA(cudaMemcpyAsync(Wm.p, Sd.p, sizeof(double) * PP, cudaMemcpyDeviceToDevice, st));
    THC_TRY(syevd(st, Wm.p, P, sv.p));
    std::vector<double> s(P);
    THC_CUDA(cudaMemcpy(s.data(), sv.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    const double smax = s[P - 1];
    if (!(smax > 0)) return Err{THC_ERR_NUMERIC, "metric S has no positive eigenvalue"};
    int k0 = 0;
    while (k0 < P && !(s[k0] > cutoff * smax)) ++k0;
    r = P - k0;
    DBuf<double> X, M, tmpPr;
    THC_TRY(X.alloc((size_t)P * r));
    k_half_inverse<<<nb((long long)P * r), 256, 0, st>>>(Wm.p, sv.p, P, k0, r, X.p);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    // M = X^T F X, eigenvectors W:  C = X W
    THC_TRY(tmpPr.alloc((size_t)P * r));
    THC_TRY(M.alloc((size_t)r * r));
    THC_TRY(mm(st, P, r, P, rm64(F.p, P), rm64(X.p, r), tmpPr.p, r, 1, 0));
    THC_TRY(mm(st, r, r, P, tr64(X.p, r), rm64(tmpPr.p, r), M.p, r, 1, 0));
    k_symmetrize<<<nb((long long)r * r), 256, 0, st>>>(M.p, r);
    count_launches(1);
    THC_TRY(e.alloc(r));
    THC_TRY(syevd(st, M.p, r, e.p));
    DBuf<double> W;
    THC_TRY(W.alloc((size_t)r * r));
    k_colmajor_to_rowmajor<<<nb((long long)r * r), 256, 0, st>>>(M.p, r, W.p);
    count_launches(1);
    THC_TRY(C.alloc((size_t)P * r));
    THC_TRY(mm(st, P, r, r, rm64(X.p, r), rm64(W.p, r), C.p, r, 1, 0));
    THC_TRY(SC.alloc((size_t)P * r));
    THC_TRY(mm(st, P, r, P, rm64(Sd.p, P), rm64(C.p, r), SC.p, r, 1, 0));
    len = (long long)o * v + (long long)r * r;
    THC_TRY(Zc.alloc(PP));
    THC_TRY(tmp.alloc((size_t)P * r));
    THC_TRY(sq.alloc((size_t)r * r));
    THC_TRY(x.alloc(len));
    THC_TRY(xnew.alloc(len));
    THC_TRY(step.alloc(len));
    THC_TRY(red.alloc(1024));
    THC_TRY(dots.alloc(64));
    THC_CUDA(cudaStreamSynchronize(st));
    return Err{};
}

template <typename T>
Err Solver::run(Engine<T>& eng, const thc_solve_opts& opts, double* Zc_io, double* t1_io,
                thc_report* rep, Mlp* mlp) {
    cudaStream_t st = eng.st;
    const auto t0 = std::chrono::steady_clock::now();
    const long long PP = (long long)P * P, ov = (long long)o * v, rr = (long long)r * r;
    const int m = std::max(0, std::min(opts.diis_n, 32));
    double energy = 0, norm = 0, e_prev = 0;
    bool converged = false;
    int it = 0, it0 = 0;
    const int max_iter = opts.max_iter > 0 ? opts.max_iter : 100;
    // learned preconditioner and training-pair recording
    const bool use_mlp = opts.use_mlp && mlp;
    const long long nrec = std::max(0, opts.record_pairs);
    double resume_last_norm = 0, resume_rho = 1;
    if (opts.resume) {
        // Continue where the last plain run stopped: x, the DIIS history and
        // the iteration count are kept; Zc_io and t1_io are outputs only.
        if (!resumable) return Err{THC_ERR_ARG, "thc_solve: no stopped solve to resume"};
        if (use_mlp || nrec > 0)
            return Err{THC_ERR_ARG, "thc_solve: resume is for plain Jacobi + DIIS solves"};
        if (m != m_done) return Err{THC_ERR_ARG, "thc_solve: resume with a different diis_n"};
        it0 = it_done;
        e_prev = e_prev_done;
        resume_last_norm = last_norm_done;
        resume_rho = rho_done;
    } else {
        if (m > 0 && hx.n < (size_t)m * len) {
            THC_TRY(hx.alloc((size_t)m * len));
            THC_TRY(he.alloc((size_t)m * len));
        }
        nhist = 0;
        head = 0;
        B.assign((size_t)std::max(m, 1) * std::max(m, 1), 0.0);
        // Start point: t1 and T = (S C)^T Zc (S C).
        THC_CUDA(cudaMemcpyAsync(x.p, t1_io, sizeof(double) * ov, cudaMemcpyDefault, st));
        THC_CUDA(cudaMemcpyAsync(Zc.p, Zc_io, sizeof(double) * PP, cudaMemcpyDefault, st));
        THC_TRY(eng.check_sym(Zc.p, P, 1e-12, "Zc"));
        THC_TRY(mm(st, P, r, P, rm64(Zc.p, P), rm64(SC.p, r), tmp.p, r, 1, 0));
        THC_TRY(mm(st, r, r, P, tr64(SC.p, r), rm64(tmp.p, r), x.p + ov, r, 1, 0));
        k_symmetrize<<<nb(rr), 256, 0, st>>>(x.p + ov, r);
        count_launches(1);
    }
    resumable = false;
    if (use_mlp || nrec > 0) {
        if (xprev.n < (size_t)len) {
            THC_TRY(xprev.alloc(len));
            THC_TRY(saved_x.alloc(len));
            THC_TRY(saved_j.alloc(len));
            THC_TRY(dprev.alloc(len));
            THC_TRY(smlp.alloc(len));
        }
    }
    if (use_mlp && feat.n < (size_t)len * kMlpFeatures) {
        THC_TRY(feat.alloc((size_t)len * kMlpFeatures));
        THC_TRY(jjb.alloc(len));
        THC_TRY(yb.alloc(len));
    }
    n_rec = 0;
    // Pairs per iteration: nrec doubles elements and a quarter as many
    // singles elements (all of them if there are fewer).
    const long long nrec1 = nrec > 0 ? std::min<long long>(ov, (nrec + 3) / 4) : 0;
    const long long nrec_it = nrec + nrec1;
    if (nrec > 0 && cap_rec < nrec_it * max_iter) {
        cap_rec = nrec_it * max_iter;
        THC_TRY(recX.alloc((size_t)cap_rec * kMlpFeatures));
        THC_TRY(recJ.alloc(cap_rec));
        THC_TRY(recT.alloc(cap_rec));
        THC_TRY(recTk.alloc(cap_rec));
        THC_TRY(recS.alloc(cap_rec));
        THC_TRY(recIdx.alloc(cap_rec));
    }
    std::vector<long long> hidx(nrec_it);
    unsigned long long rng = 0x2545F4914F6CDD1DULL ^ (unsigned long long)opts.record_seed;
    bool have_prev = false, last_was_mlp = false, mlp_off = false;
    double last_norm = resume_last_norm, rho_plain = resume_rho;
    int saved_slot = -1, n_acc = 0, n_rej = 0;
    // DIIS history: store (x, e) in slot and refresh that row of B.
    auto diis_store = [&](int slot, const double* xv, const double* ev) -> Err {
        THC_CUDA(cudaMemcpyAsync(hx.p + (long long)slot * len, xv, sizeof(double) * len,
                                 cudaMemcpyDeviceToDevice, st));
        THC_CUDA(cudaMemcpyAsync(he.p + (long long)slot * len, ev, sizeof(double) * len,
                                 cudaMemcpyDeviceToDevice, st));
        k_multidot<<<m, 256, 0, st>>>(he.p, he.p + (long long)slot * len, len, dots.p);
        count_launches(1);
        THC_CUDA(cudaGetLastError());
        std::vector<double> row(m);
        THC_CUDA(cudaMemcpyAsync(row.data(), dots.p, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        THC_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < nhist; ++k) {
            B[(size_t)slot * m + k] = row[k];
            B[(size_t)k * m + slot] = row[k];
        }
        return Err{};
    };
    // x = DIIS extrapolation of the stored pairs, or `fallback` if there is
    // too little history or the DIIS system is singular.
    auto diis_extrapolate = [&](const double* fallback) -> Err {
        std::vector<double> c;
        std::vector<double> Bsub((size_t)nhist * nhist);
        for (int i = 0; i < nhist; ++i)
            for (int j = 0; j < nhist; ++j) Bsub[(size_t)i * nhist + j] = B[(size_t)i * m + j];
        if (nhist >= 2 && diis_coefficients(Bsub, nhist, c)) {
            THC_CUDA(cudaMemcpyAsync(dots.p, c.data(), sizeof(double) * nhist,
                                     cudaMemcpyHostToDevice, st));
            k_combine<<<nb(len), 256, 0, st>>>(hx.p, dots.p, nhist, len, x.p);
            count_launches(1);
            THC_CUDA(cudaGetLastError());
        } else {
            THC_CUDA(cudaMemcpyAsync(x.p, fallback, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
        }
        return Err{};
    };
    for (it = it0 + 1; it <= it0 + max_iter; ++it) {
        // Zc = C T C^T
        THC_TRY(mm(st, P, r, r, rm64(C.p, r), rm64(x.p + ov, r), tmp.p, r, 1, 0));
        THC_TRY(mm(st, P, P, r, rm64(tmp.p, r), tr64(C.p, r), Zc.p, P, 1, 0));
        k_symmetrize<<<nb(PP), 256, 0, st>>>(Zc.p, P);
        count_launches(1);
        THC_CUDA(cudaGetLastError());
        THC_TRY(eng.set_state(Zc.p, x.p));
        THC_TRY(eng.residual_dev(true));
        THC_TRY(eng.prof_collect());
        THC_TRY(eng.check_timeout());
        // sigma_q = C^T sigma C
        THC_TRY(mm(st, P, r, P, rm64(eng.sig.p, P), rm64(C.p, r), tmp.p, r, 1, 0));
        THC_TRY(mm(st, r, r, P, tr64(C.p, r), rm64(tmp.p, r), sq.p, r, 1, 0));
        k_multidot<<<1, 256, 0, st>>>(eng.sig1.p, eng.sig1.p, ov, dots.p);
        count_launches(1);
        k_multidot<<<1, 256, 0, st>>>(sq.p, sq.p, rr, dots.p + 1);
        THC_CUDA(cudaGetLastError());
        double h[4];
        THC_CUDA(cudaMemcpyAsync(h, dots.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        THC_CUDA(cudaMemcpyAsync(h + 2, eng.en.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        THC_CUDA(cudaStreamSynchronize(st));
        norm = std::sqrt(h[0] + h[1]);
        energy = h[2] + h[3];
        if (!std::isfinite(norm) || !std::isfinite(energy))
            return Err{THC_ERR_NUMERIC, "solver diverged (non-finite residual)"};
        if (opts.history) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            opts.history[3 * (it - it0 - 1) + 0] = energy;
            opts.history[3 * (it - it0 - 1) + 1] = norm;
            opts.history[3 * (it - it0 - 1) + 2] = el;
        }
        if (opts.verbose)
            fprintf(stderr, "thc_solve it %3d  E = %.12f  |r| = %.3e\n", it, energy, norm);
        if (last_was_mlp) {
            last_was_mlp = false;
            // A proposal stands only if the residual norm drops, and by at
            // least the factor the last plain Jacobi + DIIS iteration achieved.
            const bool accept = opts.mlp_accept == 2 ||
                                (opts.mlp_accept == 1 ? norm < last_norm
                                                      : norm < last_norm * std::min(1.0, rho_plain));
            if (accept) {
                ++n_acc;
            } else {
                // Rejected: replace the proposal in the DIIS history by the
                // Jacobi step from the same point and continue from the
                // plain iterate.  Two rejections switch proposals off.
                ++n_rej;
                if (n_rej >= 2) mlp_off = true;
                k_add<<<nb(len), 256, 0, st>>>(saved_x.p, saved_j.p, len, xnew.p);
                count_launches(1);
                THC_CUDA(cudaGetLastError());
                if (m > 0 && saved_slot >= 0) {
                    THC_TRY(diis_store(saved_slot, xnew.p, saved_j.p));
                    THC_TRY(diis_extrapolate(xnew.p));
                } else {
                    THC_CUDA(cudaMemcpyAsync(x.p, xnew.p, sizeof(double) * len,
                                             cudaMemcpyDeviceToDevice, st));
                }
                THC_CUDA(cudaMemcpyAsync(xprev.p, saved_x.p, sizeof(double) * len,
                                         cudaMemcpyDeviceToDevice, st));
                continue;
            }
        } else if (it > 1 && last_norm > 0) {
            rho_plain = norm / last_norm;
        }
        const bool de_ok = opts.e_tol <= 0 || (it > 1 && std::fabs(energy - e_prev) < opts.e_tol);
        e_prev = energy;
        if (norm < opts.r_tol && de_ok) {
            converged = true;
            break;
        }
        k_jacobi<<<nb(len), 256, 0, st>>>(eng.sig1.p, sq.p, epsd.p, e.p, o, v, r, x.p,
                                           step.p, xnew.p);
        count_launches(1);
        THC_CUDA(cudaGetLastError());
        bool mlp_used = false;
        if ((nrec > 0 || use_mlp) && it >= 2) {
            // scales of this iteration's singles and doubles Jacobi steps,
            // previous step
            k_multidot<<<1, 256, 0, st>>>(step.p, step.p, ov, dots.p + 7);
            k_multidot<<<1, 256, 0, st>>>(step.p + ov, step.p + ov, rr, dots.p + 8);
            k_sub<<<nb(len), 256, 0, st>>>(x.p, xprev.p, len, dprev.p);
            count_launches(3);
            THC_CUDA(cudaGetLastError());
            double ss[2] = {0, 0};
            THC_CUDA(cudaMemcpyAsync(ss, dots.p + 7, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
            THC_CUDA(cudaStreamSynchronize(st));
            const double sc1 = std::max(std::sqrt(ss[0] / (double)ov), 1e-300);
            const double sc = std::max(std::sqrt(ss[1] / (double)rr), 1e-300);
            const double lr = std::log10(std::max(norm, 1e-300));
            const double* dp = have_prev ? dprev.p : nullptr;
            if (nrec > 0 && n_rec + nrec_it <= cap_rec) {
                for (long long k = 0; k < nrec_it; ++k) {
                    rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17;
                    hidx[k] = k < nrec ? ov + (long long)(rng % (unsigned long long)rr)
                                       : (long long)(rng % (unsigned long long)ov);
                }
                long long* di = recIdx.p + n_rec;
                THC_CUDA(cudaMemcpyAsync(di, hidx.data(), sizeof(long long) * nrec_it,
                                         cudaMemcpyHostToDevice, st));
                THC_CUDA(mlp_features(eng.sig1.p, epsd.p, sq.p, e.p, x.p, dp, di, nrec_it, o, v, r,
                                      sc1, sc, lr, recX.p + n_rec * kMlpFeatures, recJ.p + n_rec,
                                      st));
                k_gather64<<<nb(nrec_it), 256, 0, st>>>(x.p, di, nrec_it, recTk.p + n_rec);
                k_fill64<<<nb(nrec), 256, 0, st>>>(recS.p + n_rec, nrec, sc);
                k_fill64<<<nb(nrec1), 256, 0, st>>>(recS.p + n_rec + nrec, nrec1, sc1);
                count_launches(3);
                THC_CUDA(cudaGetLastError());
                // hidx is reused next iteration: the copy must finish first
                THC_CUDA(cudaStreamSynchronize(st));
                n_rec += nrec_it;
            }
            if (use_mlp && !mlp_off) {
                THC_CUDA(mlp_features(eng.sig1.p, epsd.p, sq.p, e.p, x.p, dp, nullptr, len, o, v,
                                      r, sc1, sc, lr, feat.p, jjb.p, st));
                // Rows are independent: at most 2^20 per pass bounds the
                // network's activation buffers (4 x rows x width floats).
                const long long chunk = 1LL << 20;
                for (long long r0 = 0; r0 < len; r0 += chunk)
                    THC_TRY(mlp->forward(feat.p + r0 * kMlpFeatures, std::min(chunk, len - r0),
                                         yb.p + r0));
                THC_CUDA(mlp_apply(eng.sig1.p, epsd.p, sq.p, e.p, yb.p, o, v, r,
                                   opts.mlp_blocks > 0 ? opts.mlp_blocks : 3, smlp.p, st));
                k_add<<<nb(len), 256, 0, st>>>(x.p, smlp.p, len, xnew.p);
                count_launches(1);
                THC_CUDA(cudaGetLastError());
                mlp_used = true;
            }
        }
        if (use_mlp || nrec > 0) {
            THC_CUDA(cudaMemcpyAsync(saved_x.p, x.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
            THC_CUDA(cudaMemcpyAsync(saved_j.p, step.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
            THC_CUDA(cudaMemcpyAsync(xprev.p, x.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
            have_prev = true;
        }
        // DIIS error vector = the step actually taken: the proposal replaces
        // the Jacobi step when one is made.
        if (mlp_used)
            THC_CUDA(cudaMemcpyAsync(step.p, smlp.p, sizeof(double) * len,
                                     cudaMemcpyDeviceToDevice, st));
        last_norm = norm;
        last_was_mlp = mlp_used;
        saved_slot = -1;
        if (m > 0) {
            const int slot = head;
            saved_slot = slot;
            head = (head + 1) % m;
            nhist = std::min(nhist + 1, m);
            THC_TRY(diis_store(slot, xnew.p, step.p));
            THC_TRY(diis_extrapolate(xnew.p));
        } else {
            THC_CUDA(cudaMemcpyAsync(x.p, xnew.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
        }
    }
    // Write back the last evaluated point.
    THC_CUDA(cudaMemcpyAsync(Zc_io, Zc.p, sizeof(double) * PP, cudaMemcpyDefault, st));
    THC_CUDA(cudaMemcpyAsync(t1_io, eng.t1d.p, sizeof(double) * ov, cudaMemcpyDefault, st));
    THC_CUDA(cudaStreamSynchronize(st));
    if (converged && n_rec > 0) {
        k_targets<<<nb(n_rec), 256, 0, st>>>(x.p, recIdx.p, recTk.p, recS.p, n_rec, recT.p);
        count_launches(1);
        THC_CUDA(cudaGetLastError());
        THC_CUDA(cudaStreamSynchronize(st));
    } else {
        n_rec = 0;
    }
    if (!converged && !use_mlp && nrec == 0) {
        resumable = true;
        it_done = it0 + max_iter;
        m_done = m;
        e_prev_done = e_prev;
        last_norm_done = last_norm;
        rho_done = rho_plain;
    }
    rep->iters = converged ? it : it0 + max_iter;
    rep->mlp_accepted = n_acc;
    rep->mlp_rejected = n_rej;
    rep->energy = energy;
    rep->r_norm = norm;
    rep->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!converged) return Err{THC_ERR_NOT_CONVERGED, "thc_solve reached max_iter"};
    return Err{};
}

template Err Solver::setup<double>(Engine<double>&, double);
template Err Solver::setup<float>(Engine<float>&, double);
template Err Solver::run<double>(Engine<double>&, const thc_solve_opts&, double*, double*,
                                 thc_report*, Mlp*);
template Err Solver::run<float>(Engine<float>&, const thc_solve_opts&, double*, double*,
                                thc_report*, Mlp*);

namespace {
struct StateHeader {
    unsigned long long magic;
    int P, r, o, v, m, nhist, head, it_done;
    double e_prev, last_norm, rho;
    long long len;
};
constexpr unsigned long long kStateMagic = 0x54484353544154ULL;   // "THCSTAT"
}  // namespace

size_t Solver::state_bytes() const {
    const size_t m = (size_t)m_done;
    return sizeof(StateHeader) + sizeof(double) * ((size_t)len + 2 * m * len + m * m);
}

Err Solver::state_save(void* buf, size_t bytes, cudaStream_t st) const {
    if (!resumable) return Err{THC_ERR_ARG, "no stopped plain solve to save"};
    if (!buf || bytes < state_bytes()) return Err{THC_ERR_ARG, "state buffer too small"};
    StateHeader h{kStateMagic, P, r, o, v, m_done, nhist, head, it_done, e_prev_done,
                  last_norm_done, rho_done, len};
    unsigned char* q = static_cast<unsigned char*>(buf);
    std::memcpy(q, &h, sizeof(h));
    double* d = reinterpret_cast<double*>(q + sizeof(h));
    const size_t m = (size_t)m_done;
    THC_CUDA(cudaMemcpyAsync(d, x.p, sizeof(double) * len, cudaMemcpyDeviceToHost, st));
    if (m > 0) {
        THC_CUDA(cudaMemcpyAsync(d + len, hx.p, sizeof(double) * m * len, cudaMemcpyDeviceToHost, st));
        THC_CUDA(cudaMemcpyAsync(d + len + m * len, he.p, sizeof(double) * m * len,
                                 cudaMemcpyDeviceToHost, st));
    }
    THC_CUDA(cudaStreamSynchronize(st));
    if (m > 0) std::memcpy(d + len + 2 * m * len, B.data(), sizeof(double) * m * m);
    return Err{};
}

Err Solver::state_load(const void* buf, size_t bytes, cudaStream_t st) {
    if (!buf || bytes < sizeof(StateHeader)) return Err{THC_ERR_ARG, "state buffer too small"};
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic) return Err{THC_ERR_ARG, "not a solver state"};
    if (h.P != P || h.r != r || h.o != o || h.v != v || h.len != len || h.m < 0 || h.m > 32 ||
        h.nhist < 0 || h.nhist > h.m || h.head < 0 || (h.m > 0 && h.head >= h.m))
        return Err{THC_ERR_ARG, "solver state of another system or basis"};
    const size_t m = (size_t)h.m;
    if (bytes < sizeof(StateHeader) + sizeof(double) * ((size_t)len + 2 * m * len + m * m))
        return Err{THC_ERR_ARG, "state buffer too small"};
    const double* d =
        reinterpret_cast<const double*>(static_cast<const unsigned char*>(buf) + sizeof(h));
    if (m > 0 && hx.n < m * len) {
        THC_TRY(hx.alloc(m * len));
        THC_TRY(he.alloc(m * len));
    }
    THC_CUDA(cudaMemcpyAsync(x.p, d, sizeof(double) * len, cudaMemcpyHostToDevice, st));
    if (m > 0) {
        THC_CUDA(cudaMemcpyAsync(hx.p, d + len, sizeof(double) * m * len, cudaMemcpyHostToDevice, st));
        THC_CUDA(cudaMemcpyAsync(he.p, d + len + m * len, sizeof(double) * m * len,
                                 cudaMemcpyHostToDevice, st));
    }
    THC_CUDA(cudaStreamSynchronize(st));
    B.assign(std::max<size_t>(m, 1) * std::max<size_t>(m, 1), 0.0);
    if (m > 0) std::memcpy(B.data(), d + len + 2 * m * len, sizeof(double) * m * m);
    nhist = h.nhist;
    head = h.head;
    m_done = h.m;
    it_done = h.it_done;
    e_prev_done = h.e_prev;
    last_norm_done = h.last_norm;
    rho_done = h.rho;
    resumable = true;
    return Err{};
}

Err Solver::pairs(float* X, float* j, float* t, long long max_n, long long* n_out,
                  cudaStream_t st) {
    const long long n = std::min(n_rec, max_n);
    if (n > 0) {
        if (X) THC_CUDA(cudaMemcpyAsync(X, recX.p, sizeof(float) * n * kMlpFeatures, cudaMemcpyDefault, st));
        if (j) THC_CUDA(cudaMemcpyAsync(j, recJ.p, sizeof(float) * n, cudaMemcpyDefault, st));
        if (t) THC_CUDA(cudaMemcpyAsync(t, recT.p, sizeof(float) * n, cudaMemcpyDefault, st));
        THC_CUDA(cudaStreamSynchronize(st));
    }
    *n_out = n_rec;
    return Err{};
}

}  // namespace thc
