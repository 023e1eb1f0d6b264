// Residual engine: factorised evaluation of the projected THC-RR-CCSD
// residual (Algorithms 1-10 of the paper) on one GPU.
//
// Notation: y_o = Y[0:o], y_v = Y[o:n] (amplitude collocation, Eq. 23),
// x_o, x_v likewise for the ERI grid (Eq. 17), T = Zc the THC core,
// o^XY = y_o^T y_o, v^XY = y_v^T y_v (Alg. 1 lines 1-2), S = o * v (Eq. 10).
// Dressed Cholesky blocks per vector A (Eqs. 25-27, C = 1 in the MO basis):
//   L^_oo = L_oo + L_ov t1^T,  L^_vv = L_vv - t1^T L_ov,
//   L^_vo = L_vo + L_vv t1^T - t1^T L^_oo,  L^_ov = L_ov.
#include <cstring>
#include <type_traits>

#include "engine.cuh"

namespace thc {

namespace {

template <typename T>
__global__ void k_wen_acc(const T* E, int P, int nb, double* acc) {
    const long long PP = (long long)P * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < PP;
         idx += (long long)gridDim.x * blockDim.x) {
        const int Y = (int)(idx / P), Z = (int)(idx % P);
        double s = 0;
        for (int a = 0; a < nb; ++a)
            s += (double)E[a * PP + (long long)Z * P + Y] * (double)E[a * PP + idx];
        acc[idx] -= s;
    }
}

template <typename T>
__global__ void k_outer_acc(const T* Acols, int P, int K, double* acc, double scale) {
    const long long PP = (long long)P * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < PP;
         idx += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(idx / P), Y = (int)(idx % P);
        double s = 0;
        for (int a = 0; a < K; ++a)
            s += (double)Acols[(long long)X * K + a] * (double)Acols[(long long)Y * K + a];
        acc[idx] += scale * s;
    }
}

__global__ void k_asym(const double* a, int n, unsigned long long* out) {
    // out[0] = bits of max |a - a^T|, out[1] = bits of max |a|, out[2] = # non-finite
    const long long nn = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        const double x = a[idx];
        if (!isfinite(x)) { atomicAdd(&out[2], 1ULL); continue; }
        const double d = fabs(x - a[(long long)j * n + i]);
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(isfinite(d) ? d : 0.0));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(fabs(x)));
    }
}

}  // namespace

template <typename T>
Err Engine<T>::check_timeout() {
    if (!tcerr.p) return Err{};
    int h = 0;
    THC_CUDA(cudaMemcpyAsync(&h, tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    THC_CUDA(cudaStreamSynchronize(st));
    if (h) {
        THC_CUDA(cudaMemsetAsync(tcerr.p, 0, sizeof(int), st));
        return Err{THC_ERR_TIMEOUT, "a tensor-core kernel's bounded wait expired"};
    }
    return Err{};
}

template <typename T>
Err Engine<T>::check_sym(const double* a, int nn_, double rel, const char* what) {
    unsigned long long h[3];
    THC_CUDA(cudaMemsetAsync(chk.p, 0, 3 * sizeof(unsigned long long), st));
    const long long tot = (long long)nn_ * nn_;
    k_asym<<<(unsigned)std::min<long long>((tot + 255) / 256, 152 * 32), 256, 0, st>>>(a, nn_, chk.p);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    THC_CUDA(cudaMemcpyAsync(h, chk.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    THC_CUDA(cudaStreamSynchronize(st));
    if (h[2]) return Err{THC_ERR_NUMERIC, std::string(what) + " has non-finite entries"};
    double asym, amax;
    memcpy(&asym, &h[0], 8);
    memcpy(&amax, &h[1], 8);
    if (asym > rel * amax) return Err{THC_ERR_ARG, std::string(what) + " is not symmetric"};
    return Err{};
}

template <typename T>
Err Engine<T>::check_finite(const double* a, long long count, const char* what) {
    int bad = 0;
    THC_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    THC_CUDA(any_nonfinite(a, count, flag.p, st));
    THC_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    THC_CUDA(cudaStreamSynchronize(st));
    if (bad) return Err{THC_ERR_NUMERIC, std::string(what) + " has non-finite entries"};
    return Err{};
}

template <typename T>
void Engine<T>::seg_begin(int step) {
    step_now = step;
    // NVTX range per step (visible to ncu's NVTX filters and other tools)
    if (nvtx_open) nvtxRangePop();
    nvtxRangePushA(thc_step_name(step));
    nvtx_open = true;
    if (!prof.on) return;
    if (prof.cur >= 0) prof_close();
    cudaEvent_t e = prof.next_event();
    cudaEventRecord(e, st);
    prof.marks.push_back({step, {prof.used - 1, -1}});
    prof.cur = step;
}

template <typename T>
void Engine<T>::seg_end() {
    step_now = -1;
    if (nvtx_open) {
        nvtxRangePop();
        nvtx_open = false;
    }
    prof_close();
}

template <typename T>
void Engine<T>::prof_close() {
    if (!prof.on || prof.cur < 0) return;
    cudaEvent_t e = prof.next_event();
    cudaEventRecord(e, st);
    prof.marks.back().second.second = prof.used - 1;
    prof.cur = -1;
}

template <typename T>
Err Engine<T>::prof_collect() {
    if (!prof.on) return Err{};
    seg_end();
    THC_CUDA(cudaStreamSynchronize(st));
    for (auto& m : prof.marks) {
        if (m.second.second < 0) continue;
        float t = 0;
        THC_CUDA(cudaEventElapsedTime(&t, prof.pool[m.second.first], prof.pool[m.second.second]));
        prof.ms[m.first] += t;
        prof.launches[m.first] += 1;
    }
    prof.marks.clear();
    prof.used = 0;
    prof.residuals += 1;
    prof.kernel_launches = launches() - prof.launch_base;
    return Err{};
}

template <typename T>
static View<T> rm(const T* p, long long ld) { return View<T>{p, ld, 1}; }
template <typename T>
static View<T> tr(const T* p, long long ld) { return View<T>{p, 1, ld}; }

template <typename T>
Err Engine<T>::mm(int M, int N, int Kd, View<T> A, View<T> B, T* C, long long ldc,
                  double alpha, double beta, int batch, long long sAb, long long sBb,
                  long long sCb, bool reduce) {
    Gemm<T> g;
    g.M = M; g.N = N; g.K = Kd; g.batch = batch;
    g.A = A; g.B = B; g.sAb = sAb; g.sBb = sBb;
    g.C = C; g.ldc = ldc; g.sCb = sCb;
    g.alpha = alpha; g.beta = beta; g.reduce = reduce;
    g.ws = splitk.p; g.ws_elems = splitk.n;
    const double fl = 2.0 * M * N * (double)Kd * batch;
    if (prof.on && prof.cur >= 0) prof.flops[prof.cur] += fl;
    const char* why = nullptr;   // why a large product stays on the CUDA cores
    if constexpr (std::is_same<T, float>::value) {
        // Large products go to the tensor cores; the rest stays on the CUDA
        // cores (also if the packed operands do not fit the workspace).
        const int tcp = tcws.buf ? step_tcp() : 0;
        if (tcp > 0 && fl >= 3.0e7 && Kd >= 16) {
            cudaError_t e = gemm_tc(g, tcws, tcp, st, &pcache);
            if (e == cudaSuccess) return Err{};
            if (e != cudaErrorMemoryAllocation) THC_CUDA(e);
            why = "workspace";
        } else if (tcp > 0 && fl >= 3.0e7) {
            why = "K < 16";
        }
    } else {
        // float64 products by exact integer slices on the tensor cores, when
        // the estimated time beats the CUDA cores (1 TFLOP/s): 36 slice-pair
        // products at the 0.85 PFLOP/s of bf16 products the fused kernel
        // reaches on large shapes, slicing (8 + 8 bytes read, 16 written per
        // operand element), the float64 tile written once, 5 launches.
        const double out = (double)M * N * (reduce ? 1 : batch);
        const double opnd = ((double)M + N) * Kd * batch;
        const double t_tc = 36.0 * fl / 0.85e15 + opnd * 32.0 / 5e12 + out * 8.0 / 5e12 +
                            5.0 * 5e-6;
        const bool use_tc = step_f64tc();
        if (use_tc && fl >= 3.0e7 && Kd >= 16 && t_tc < fl / 1.0e12) {
            cudaError_t e = gemm_f64_tc(g, f64ws, st);
            if (e == cudaSuccess) return Err{};
            if (e != cudaErrorMemoryAllocation) THC_CUDA(e);
            why = "workspace";
        } else if (use_tc && fl >= 3.0e7) {
            why = Kd < 16 ? "K < 16" : "cost model";
        }
    }
    if (why && debug_products())
        fprintf(stderr, "thc: product M=%d N=%d K=%d batch=%d%s (%.3g flop) on the CUDA cores: %s\n",
                M, N, Kd, batch, reduce ? " reduced" : "", fl, why);
    THC_CUDA(gemm_simt(g, st));
    return Err{};
}

template <typename T>
Err Engine<T>::dress(const T* oo_, const T* ov_, const T* vv_, int nb, T* out_oo,
                     T* out_vv, T* out_vo) {
    const T* tp = t1.p;
    // L^_oo = L_oo + L_ov t1^T
    THC_CUDA(cudaMemcpyAsync(out_oo, oo_, sizeof(T) * nb * o * o, cudaMemcpyDeviceToDevice, st));
    THC_TRY(mm(o, o, v, rm(ov_, v), tr(tp, v), out_oo, o, 1, 1, nb, (long long)o * v, 0,
               (long long)o * o));
    // L_vv from its packed lower triangles (vv_), still undressed
    THC_CUDA(unpack_vv(vv_, nb, v, out_vv, st));
    // L^_vo = L_ov^T + L_vv t1^T - t1^T L^_oo
    THC_CUDA(transpose_batched(ov_, out_vo, nb, o, v, st));
    THC_TRY(mm(v, o, v, rm(out_vv, v), tr(tp, v), out_vo, o, 1, 1, nb, (long long)v * v, 0,
               (long long)v * o));
    THC_TRY(mm(v, o, o, tr(tp, v), rm(out_oo, o), out_vo, o, -1, 1, nb, 0, (long long)o * o,
               (long long)v * o));
    // L^_vv = L_vv - t1^T L_ov
    THC_TRY(mm(v, v, o, tr(tp, v), rm(ov_, v), out_vv, v, -1, 1, nb, 0, (long long)o * v,
               (long long)v * v));
    return Err{};
}

// The T1-dressed Fock matrix F^ = h^ + 2 J(L^) - X(L^) (Eqs. 24-27 applied to the
// canonical Fock operator f = diag(eps) with h backed out) written without
// its large cancelling parts.  With t the n x n matrix holding t_i^a in block
// (a, i), L^ = (1 - t) L (1 + t), and t t = 0:
//   J(L^) = dress(J(L)) + sum_A delta^A L^^A,   delta^A = sum_ia t_i^a L_ia^A,
//   X(L^) = dress(X(L)) + sum_A L^^A t L^^A,
// so that  F^ = dress(f) + 2 sum_A delta^A L^^A - sum_A L^^A t L^^A  with
// dress(f) = f + (eps_a - eps_i) t_i^a in block (a, i).  Every term but f is
// of order t1, so the float32 engine keeps its relative precision where the
// direct form subtracts Coulomb sums of order o times (pp|qq).
// This routine accumulates, for the nb dressed vectors of a slab,
//   J_pq += sum_A delta^A L^_pq^A,   X_pq += sum_A sum_ai L^_pa^A t_i^a L^_iq^A.
template <typename T>
Err Engine<T>::fock_slab(int nb, const T* Loo_, const T* Lov_, const T* Lvo_, const T* Lvv_) {
    const long long oo2 = (long long)o * o, ov = (long long)o * v, vv2 = (long long)v * v;
    const T* tp = t1.p;
    // delta^A = sum_ia L_ia^A t_i^a
    THC_TRY(mm(nb, 1, (int)ov, rm(Lov_, ov), View<T>{tp, 1, 0}, dtr.p, 1, 1, 0));
    View<T> d{dtr.p, 0, 1};
    THC_TRY(mm(1, (int)oo2, nb, d, rm(Loo_, oo2), Joo.p, oo2, 1, 1));
    THC_TRY(mm(1, (int)ov, nb, d, rm(Lov_, ov), Jov.p, ov, 1, 1));
    THC_TRY(mm(1, (int)ov, nb, d, rm(Lvo_, ov), Jvo.p, ov, 1, 1));
    THC_TRY(mm(1, (int)vv2, nb, d, rm(Lvv_, vv2), Jvv.p, vv2, 1, 1));
    // W_o^A = L^_ov^A t1^T (o x o),  W_v^A = L^_vv^A t1^T (v x o)
    THC_TRY(mm(o, o, v, rm(Lov_, v), tr(tp, v), Wfo.p, o, 1, 0, nb, ov, 0, oo2));
    THC_TRY(mm(v, o, v, rm(Lvv_, v), tr(tp, v), Wfv.p, o, 1, 0, nb, vv2, 0, ov));
    THC_TRY(mm(o, o, o, rm(Wfo.p, o), rm(Loo_, o), Xoo.p, o, 1, 1, nb, oo2, oo2, 0, true));
    THC_TRY(mm(o, v, o, rm(Wfo.p, o), rm(Lov_, v), Xov.p, v, 1, 1, nb, oo2, ov, 0, true));
    THC_TRY(mm(v, o, o, rm(Wfv.p, o), rm(Loo_, o), Xvo.p, o, 1, 1, nb, ov, oo2, 0, true));
    THC_TRY(mm(v, v, o, rm(Wfv.p, o), rm(Lov_, v), Xvv.p, v, 1, 1, nb, ov, ov, 0, true));
    return Err{};
}

// D_ia = sum_kc (2 t_ik^ac - t_ik^ca) M_kc for nb matrices M (o x v):
// D = y_o (2 diag(T a) - T o E) y_v^T,  a^X = sum_ia y_i^X y_a^X M_ia,
// E^YZ = sum_kc y_c^Y y_k^Z M_kc   (Alg. 8 lines 6-9, Alg. 10 lines 1-8).
template <typename T>
Err Engine<T>::d_operator(const T* Mv, int nb, T* Dout) {
    const long long ov = (long long)o * v, oP = (long long)o * P, PP = (long long)P * P;
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    THC_TRY(mm(o, P, v, rm(Mv, v), rm(yv, P), M3.p, P, 1, 0, nb, ov, 0, oP));
    THC_CUDA(diag_reduce(yo, M3.p, o, P, nb, Ta0.p, nb, 0, st));
    THC_TRY(mm(P, nb, P, rm(Tc.p, P), rm(Ta0.p, nb), TA.p, nb, 1, 0));
    THC_TRY(mm(P, P, o, tr(M3.p, P), rm(yo, P), E.p, P, 1, 0, nb, oP, 0, PP));
    THC_CUDA(w_single(TA.p, nb, Tc.p, E.p, W.p, P, nb, st));
    THC_TRY(mm(o, P, P, rm(yo, P), rm(W.p, P), M4.p, P, 1, 0, nb, 0, PP, oP));
    THC_TRY(mm(o, v, P, rm(M4.p, P), tr(yv, P), Dout, v, 1, 0, nb, oP, 0, ov));
    return Err{};
}

template <typename T>
Err Engine<T>::init(const thc_config& cfg, const double* eps_o, const double* eps_v,
                    const double* Yh, const double* Lh, const double* xh, const double* zh,
                    cudaStream_t s) {
    THC_TRY(init_begin(cfg, eps_o, eps_v, Yh, xh, zh, s));
    if (!Lh) return Err{};   // the caller supplies the Cholesky vectors
    THC_TRY(load_cholesky(0, Kglob, Lh));
    return init_finish();
}

template <typename T>
Err Engine<T>::init_begin(const thc_config& cfg, const double* eps_o, const double* eps_v,
                          const double* Yh, const double* xh, const double* zh,
                          cudaStream_t s) {
    st = s;
    cfg0 = cfg;
    o = cfg.n_occ; v = cfg.n_vir; n = o + v; P = cfg.n_p; G = cfg.n_g; K = cfg.n_k;
    // Shard: a contiguous range of Cholesky vectors and of Alg. 6 rows X.
    Kglob = K;
    nsh = cfg.shard_count > 1 ? cfg.shard_count : 1;
    ish = nsh > 1 ? cfg.shard_index : 0;
    K0 = (int)((long long)Kglob * ish / nsh);
    K = (int)((long long)Kglob * (ish + 1) / nsh) - K0;
    x_lo = (int)((long long)P * ish / nsh);
    x_hi = (int)((long long)P * (ish + 1) / nsh);
    do_alg7 = ish == nsh - 1;
    f_terms = ish == 0;
    // Per-step arithmetic: the context's policy unless the step names its own.
    f64tc_default = std::is_same<T, double>::value && cfg.precision == THC_PREC_FP64_TC;
    for (int s_ = 0; s_ < THC_N_STEPS; ++s_) {
        int p = cfg.policy[s_];
        if (p == THC_POL_DEFAULT) {
            if (std::is_same<T, double>::value)
                p = f64tc_default ? THC_POL_FP64_TC : THC_POL_FP64;
            else
                p = cfg.tc_products == 3 ? THC_POL_BF16X3
                                         : (cfg.tc_products == 1 ? THC_POL_BF16 : THC_POL_FP32);
        }
        if (!std::is_same<T, double>::value && s_ == THC_STEP_TRIANGLE) p = THC_POL_FP32;
        pol[s_] = p;
    }
    {
        // Cholesky slab: as many vectors as the per-vector scratch budget holds
        // (six P x P intermediates dominate), at least 16.  The budget is a
        // tenth of the free device memory, between 2 and 16 GiB: fewer, longer
        // slabs mean fewer launches of the slab pass's many small products.
        const long long per = 6LL * cfg.n_p * cfg.n_p + 2LL * cfg.n_vir * cfg.n_vir +
                              8LL * (cfg.n_occ + cfg.n_vir) * cfg.n_p;
        size_t free_b = 0, total_b = 0;
        long long budget = 2LL << 30;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
            budget = std::max<long long>(budget, std::min<long long>(16LL << 30,
                                                                     (long long)(free_b / 10)));
        const long long fit = budget / (per * (long long)sizeof(T));
        kb = cfg.k_slab > 0 ? std::min(cfg.k_slab, K)
                            : (int)std::max<long long>(1, std::min<long long>(
                                  K, std::max<long long>(16, fit)));
    }
    const long long ov = (long long)o * v, vt = (long long)v * (v + 1) / 2;

    THC_TRY(flag.alloc(1));
    THC_TRY(chk.alloc(3));
    {
        DBuf<double> zd, ed;
        THC_TRY(zd.alloc((size_t)G * G));
        THC_CUDA(cudaMemcpyAsync(zd.p, zh, sizeof(double) * G * G, cudaMemcpyDefault, st));
        THC_TRY(check_sym(zd.p, G, 1e-12, "z"));
        THC_TRY(ed.alloc((size_t)n));
        THC_CUDA(cudaMemcpyAsync(ed.p, eps_o, sizeof(double) * o, cudaMemcpyDefault, st));
        THC_CUDA(cudaMemcpyAsync(ed.p + o, eps_v, sizeof(double) * v, cudaMemcpyDefault, st));
        THC_TRY(check_finite(ed.p, n, "orbital energies"));
    }
    // ---- fixed inputs
    THC_TRY(y.alloc((size_t)n * P));
    THC_TRY(x.alloc((size_t)n * G));
    THC_TRY(z.alloc((size_t)G * G));
    THC_TRY(load(Yh, y.p, (long long)n * P));
    THC_TRY(load(xh, x.p, (long long)n * G));
    THC_TRY(load(zh, z.p, (long long)G * G));
    THC_TRY(Loo.alloc((size_t)K * o * o));
    THC_TRY(Lov.alloc((size_t)K * ov));
    THC_TRY(Lvv.alloc((size_t)K * vt));

    // ---- canonical Fock operator f = diag(eps): the reference is canonical
    // Hartree-Fock, and the core Hamiltonian it implies (h = f - 2 J + X) is
    // never formed (see fock_slab).
    THC_TRY(foo.alloc((size_t)o * o));
    THC_TRY(fvv.alloc((size_t)v * v));
    THC_TRY(epsT.alloc(n));
    {
        std::vector<double> eps(n);
        THC_CUDA(cudaMemcpy(eps.data(), eps_o, sizeof(double) * o, cudaMemcpyDefault));
        THC_CUDA(cudaMemcpy(eps.data() + o, eps_v, sizeof(double) * v, cudaMemcpyDefault));
        eps_h = eps;
        std::vector<T> fo((size_t)o * o, T(0)), fv((size_t)v * v, T(0)), et(n);
        for (int i = 0; i < o; ++i) fo[(size_t)i * o + i] = (T)eps[i];
        for (int a = 0; a < v; ++a) fv[(size_t)a * v + a] = (T)eps[o + a];
        for (int p = 0; p < n; ++p) et[p] = (T)eps[p];
        THC_CUDA(cudaMemcpyAsync(foo.p, fo.data(), sizeof(T) * o * o, cudaMemcpyHostToDevice, st));
        THC_CUDA(cudaMemcpyAsync(fvv.p, fv.data(), sizeof(T) * v * v, cudaMemcpyHostToDevice, st));
        THC_CUDA(cudaMemcpyAsync(epsT.p, et.data(), sizeof(T) * n, cudaMemcpyHostToDevice, st));
        THC_CUDA(cudaStreamSynchronize(st));
    }
    loaded.assign((size_t)K, 0);
    pending = true;
    return Err{};
}

template <typename T>
Err Engine<T>::load_cholesky(int k0, int nk, const double* Lh) {
    if (!pending) return Err{THC_ERR_ARG, "the Cholesky vectors are already set"};
    if (!Lh || k0 < 0 || nk <= 0 || (long long)k0 + nk > Kglob)
        return Err{THC_ERR_ARG, "Cholesky vector range outside 0 .. K - 1"};
    const long long ov = (long long)o * v, nn = (long long)n * n,
                    vt = (long long)v * (v + 1) / 2;
    // Only the shard's own vectors [K0, K0 + K) are stored, at k - K0.
    {
        const long long lo = std::max<long long>(k0, K0);
        const long long hi = std::min<long long>((long long)k0 + nk, (long long)K0 + K);
        if (lo >= hi) return Err{};
        Lh += (lo - k0) * nn;
        k0 = (int)(lo - K0);
        nk = (int)(hi - lo);
    }
    if (!lstage.p) {
        THC_TRY(lstage.alloc((size_t)kb * nn));
        if (!std::is_same<T, double>::value) THC_TRY(lstageT.alloc((size_t)kb * nn));
    }
    // Stage kb vectors at a time and split them into their blocks (the vv
    // block as its lower triangle).
    for (int a = 0; a < nk; a += kb) {
        const int nb = std::min(kb, nk - a);
        const long long A0 = (long long)k0 + a;
        THC_CUDA(cudaMemcpyAsync(lstage.p, Lh + (long long)a * nn, sizeof(double) * nb * nn,
                                 cudaMemcpyDefault, st));
        const T* src;
        if constexpr (std::is_same<T, double>::value) {
            src = lstage.p;
        } else {
            THC_CUDA(convert(lstage.p, lstageT.p, nb * nn, st));
            src = lstageT.p;
        }
        Blocks<T> b;
        b.oo = Loo.p + A0 * o * o;
        b.ov = Lov.p + A0 * ov;
        b.vvp = Lvv.p + A0 * vt;
        THC_CUDA(split_blocks(src, nb, o, v, b, st));
    }
    THC_CUDA(cudaStreamSynchronize(st));   // the caller may reuse its buffer
    for (int k = k0; k < k0 + nk; ++k) loaded[k] = 1;
    return Err{};
}

template <typename T>
Err Engine<T>::init_finish() {
    if (!pending) return Err{THC_ERR_ARG, "no initialisation is pending"};
    for (int k = 0; k < K; ++k)
        if (!loaded[k])
            return Err{THC_ERR_ARG, "Cholesky vector " + std::to_string(k) + " was not loaded"};
    lstage.release();
    lstageT.release();
    const thc_config& cfg = cfg0;
    const long long ov = (long long)o * v, PP = (long long)P * P;
    const long long TB = (long long)sizeof(T);

    // ---- scratch
    const long long kbl = kb;
    THC_TRY(splitk.alloc((size_t)std::max<long long>(4 * PP, 1 << 22)));
    THC_TRY(Tc.alloc(PP));
    THC_TRY(Tcd.alloc(PP));
    THC_TRY(t1.alloc(ov));
    THC_TRY(t1d.alloc(ov));
    THC_TRY(sig.alloc(PP));
    THC_TRY(sig1.alloc(ov));
    THC_TRY(en.alloc(4));
    if (!std::is_same<T, double>::value) {
        THC_TRY(sigT.alloc(PP));
        THC_TRY(sig1T.alloc(ov));
    }
    THC_TRY(xoo.alloc((size_t)o * o));
    THC_TRY(xvv.alloc((size_t)v * v));
    THC_TRY(Ccross.alloc(PP));
    THC_TRY(Abar.alloc((size_t)P * K));
    THC_TRY(Q.alloc((size_t)P * K));
    THC_TRY(Wq.alloc((size_t)P * K));
    for (DBuf<T>* b : {&Joo, &Xoo, &Foo}) THC_TRY(b->alloc((size_t)o * o));
    for (DBuf<T>* b : {&Jov, &Xov, &Fov, &Jvo, &Xvo, &Fvo, &E1}) THC_TRY(b->alloc(ov));
    for (DBuf<T>* b : {&Jvv, &Xvv, &Fvv}) THC_TRY(b->alloc((size_t)v * v));
    for (DBuf<T>* b : {&ST, &E9, &V9, &O9}) THC_TRY(b->alloc(PP));
    THC_TRY(M9.alloc((size_t)n * P));
    THC_TRY(FvoT.alloc(ov));
    THC_TRY(red.alloc(std::max(1024, K + 16)));
    THC_TRY(Lh_oo.alloc(kbl * o * o));
    THC_TRY(Lh_vv.alloc(kbl * v * v));
    THC_TRY(Lh_vo.alloc(kbl * ov));
    THC_TRY(dtr.alloc(kbl));
    THC_TRY(Wfo.alloc(kbl * o * o));
    THC_TRY(Wfv.alloc(kbl * ov));
    THC_TRY(M1.alloc(kbl * o * P));
    THC_TRY(N1.alloc(kbl * v * P));
    THC_TRY(M2.alloc(kbl * v * P));
    THC_TRY(M3.alloc(kbl * o * P));
    THC_TRY(M4.alloc(kbl * o * P));
    THC_TRY(M5.alloc(kbl * o * P));
    for (DBuf<T>* b : {&Bbar, &Btil, &C1, &D1, &E, &W}) THC_TRY(b->alloc(kbl * PP));
    THC_TRY(TA.alloc(kbl * P));
    THC_TRY(Ta0.alloc(kbl * P));
    THC_TRY(D8.alloc(kbl * ov));
    THC_TRY(Mo.alloc((size_t)K * o * o));

    // ---- amplitude-factor products
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    const T* xo = x.p;
    const T* xv = x.p + (long long)o * G;
    THC_TRY(oo.alloc(PP));
    THC_TRY(vv.alloc(PP));
    THC_TRY(S.alloc(PP));
    THC_TRY(mm(P, P, o, tr(yo, P), rm(yo, P), oo.p, P, 1, 0));
    THC_TRY(mm(P, P, v, tr(yv, P), rm(yv, P), vv.p, P, 1, 0));
    THC_CUDA(hadamard2(S.p, PP, oo.p, vv.p, (const T*)nullptr, (const T*)nullptr, st));
    THC_TRY(KRy.alloc(ov * P));
    THC_CUDA(khatri_rao(yo, yv, o, v, P, KRy.p, st));

    // ---- energy weight  Wen = 2 sum_A a_A a_A^T - sum_A E_A^T o E_A   (float64)
    THC_TRY(Atil.alloc((size_t)P * K));
    THC_TRY(Wen.alloc(PP));
    THC_CUDA(cudaMemsetAsync(Wen.p, 0, PP * sizeof(double), st));
    for (int A0 = 0; A0 < K; A0 += kb) {
        int nb = std::min(kb, K - A0);
        THC_TRY(mm(o, P, v, rm(Lov.p + A0 * ov, v), rm(yv, P), M3.p, P, 1, 0, nb, ov, 0,
                   (long long)o * P));
        THC_CUDA(diag_reduce(yo, M3.p, o, P, nb, Atil.p, K, A0, st));
        THC_TRY(mm(P, P, o, tr(M3.p, P), rm(yo, P), E.p, P, 1, 0, nb, (long long)o * P, 0, PP));
        k_wen_acc<T><<<cdiv(PP, 256), 256, 0, st>>>(E.p, P, nb, Wen.p);
        count_launches(1);
        THC_CUDA(cudaGetLastError());
    }
    k_outer_acc<T><<<cdiv(PP, 256), 256, 0, st>>>(Atil.p, P, K, Wen.p, 2.0);
    count_launches(1);
    THC_CUDA(cudaGetLastError());

    // ---- Alg. 7 route.  Dense route: Kx[(ia),(jb)] = (ib|ja) =
    //      sum_J B[(i,b),J] x_j^J x_a^J, when it takes at most 16 GiB; built
    //      only by the shard that evaluates Alg. 7.
    {
        const double kx_bytes = (double)ov * ov * sizeof(T);
        alg7_dense = cfg.alg7_route == 2 ||
                     (cfg.alg7_route == 0 && kx_bytes <= 16.0 * (1LL << 30));
    }
    const bool dense_init = alg7_dense && do_alg7;
    // ---- Float64 products of init (B, U, Kx below) on the tensor cores:
    //      a workspace of at most an eighth of the free memory (24 GiB at
    //      most; larger products are cut into pieces), released before the
    //      residual's own workspace is sized.
    struct Shape { long long M, N, K, b; };
    const long long per_i = (long long)v * G;   // x o x and B elements per occupied orbital
    const int ci = dense_init ? o
                              : (int)std::max<long long>(
                                    1, std::min<long long>(o, (4LL << 30) / (2 * per_i * TB)));
    const bool init_f64tc = std::is_same<T, double>::value && f64tc_default;
    if (init_f64tc) {
        std::vector<Shape> ishapes = {{(long long)ci * v, G, G, 1}, {G, P, v, ci}};
        if (dense_init) ishapes.push_back({v, v, G, o});
        size_t sl = 0, pt = 0, ex = 0;
        for (const Shape& sh : ishapes) {
            size_t a_ = 0, b_ = 0, c_ = 0;
            gemm_f64_tc_sizes((int)sh.M, (int)sh.N, (int)sh.K, (int)sh.b, false, &a_, &b_, &c_);
            sl = std::max(sl, a_);
            pt = std::max(pt, b_);
            ex = std::max(ex, c_);
        }
        size_t cap = 24ull << 30, free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) cap = std::min(cap, free_b / 8);
        sl = std::min(sl, cap / 4 * 3 / sizeof(__nv_bfloat16));
        pt = std::min(pt, cap / 4 / sizeof(float));
        THC_TRY(f64sl.alloc(sl));
        THC_TRY(f64part.alloc(pt));
        THC_TRY(f64exp.alloc(ex));
        THC_TRY(tcerr.alloc(1));
        THC_CUDA(cudaMemsetAsync(tcerr.p, 0, sizeof(int), st));
        f64ws = F64TcWorkspace{f64sl.p, f64sl.n, f64part.p, f64part.n, f64exp.p, f64exp.n,
                               tcerr.p};
        f64tc = true;
    }

    // ---- Alg. 6 fixed parts: B_ia^I = sum_J x_i^J x_a^J z^IJ (line 2),
    //      U[i][I][Z] = sum_a B_ia^I y_a^Z, G_I^YZ = sum_i y_i^Y U[i][I][Z] (line 10)
    THC_TRY(U6.alloc((size_t)o * G * P));
    if (dense_init) {
        THC_TRY(KRx.alloc(ov * G));
        THC_CUDA(khatri_rao(xo, xv, o, v, G, KRx.p, st));
        THC_TRY(B6.alloc(ov * G));
        THC_TRY(mm((int)ov, G, G, rm(KRx.p, G), rm(z.p, G), B6.p, G, 1, 0));
        THC_TRY(mm(G, P, v, View<T>{B6.p, 1, G}, rm(yv, P), U6.p, P, 1, 0, o, (long long)v * G,
                   0, (long long)G * P));
        THC_TRY(Kx.alloc((size_t)ov * ov));
        THC_TRY(W7.alloc((size_t)P * ov));
        for (int i = 0; i < o; ++i)
            THC_TRY(mm(v, v, G, rm(KRx.p, G), tr(B6.p + (long long)i * v * G, G),
                       Kx.p + (long long)i * v * ov, ov, 1, 0, o, (long long)v * G, 0, v));
    } else {
        // x o x and B for ci occupied orbitals at a time (at most 4 GiB for
        // both): neither is ever held whole.
        THC_TRY(KRx.alloc((size_t)ci * per_i));
        THC_TRY(B6.alloc((size_t)ci * per_i));
        for (int i0 = 0; i0 < o; i0 += ci) {
            const int nc = std::min(ci, o - i0);
            THC_CUDA(khatri_rao(xo + (long long)i0 * G, xv, nc, v, G, KRx.p, st));
            THC_TRY(mm(nc * v, G, G, rm(KRx.p, G), rm(z.p, G), B6.p, G, 1, 0));
            THC_TRY(mm(G, P, v, View<T>{B6.p, 1, G}, rm(yv, P), U6.p + (long long)i0 * G * P, P,
                       1, 0, nc, (long long)v * G, 0, (long long)G * P));
        }
    }
    // B is needed only to build U (and Kx); x o x only on the dense route
    // (C^XI of the blocked route comes from its per-X intermediates).
    THC_CUDA(cudaStreamSynchronize(st));
    B6.release();
    if (!dense_init) KRx.release();
    if (init_f64tc) {
        f64sl.release();
        f64part.release();
        f64exp.release();
        f64ws = F64TcWorkspace{};
        f64tc = false;
    }

    // ---- Alg. 6 blocking.  G_I^YZ is resident when it fits; otherwise it
    //      is rebuilt per grid chunk (and per X block).  X blocks: H (x6 P^2),
    //      its packed copy for the post-products, D_a and C_i (x6 P each per
    //      orbital) take at most a quarter of the free memory (48 GiB at
    //      most); all P rows in one block when they fit, else the fewest
    //      blocks that do, rounded up to the triangle kernel's 32-row tile.
    const size_t gall_bytes = (size_t)G * PP * sizeof(T);
    const bool gall_fits = cfg.workspace_bytes == 0 ? gall_bytes <= (size_t)48 << 30
                                                    : gall_bytes <= cfg.workspace_bytes / 4;
    {
        size_t free_b = 0, total_b = 0;
        long long budget6 = cfg.workspace_bytes > 0 ? (long long)(cfg.workspace_bytes / 4)
                                                    : 48LL << 30;
        if (cfg.workspace_bytes == 0 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
            budget6 = std::min<long long>(budget6, (long long)(free_b / 4));
        const long long perX = (2 * PP + (long long)(o + v) * P) * TB;
        if (cfg.x_block6 > 0) {
            x6 = std::min(cfg.x_block6, P);
        } else if (perX * P <= budget6) {
            x6 = P;
        } else {
            const long long nblk = (perX * P + budget6 - 1) / std::max<long long>(budget6, 1);
            x6 = (int)std::min<long long>(P, ((P + nblk - 1) / nblk + 31) / 32 * 32);
        }
        // Grid points per chunk: the E and F chunks take at most 4 GB; a
        // rebuilt G chunk takes a twelfth of the free memory, 4-12 GiB (more
        // grid points per triangle launch: fewer read-modify-writes of H).
        long long icl = (4LL << 30) / (2LL * x6 * P * TB);
        if (!gall_fits) {
            long long gbudget = 4LL << 30;
            if (cfg.workspace_bytes == 0 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                gbudget = std::max<long long>(gbudget, std::min<long long>(
                                                           12LL << 30, (long long)(free_b / 12)));
            icl = std::min<long long>(icl, gbudget / (PP * TB));
        }
        ic = cfg.i_chunk > 0 ? std::min(cfg.i_chunk, G)
                             : (int)std::max<long long>(1, std::min<long long>(G, icl));
    }
    const int nblk6 = (P + x6 - 1) / x6;
    // ---- Route for Eqs. 32-33: Alg. 6 (O(N^4), triangle on the CUDA cores)
    //      or Algs. 4 and 5 (O(N^5), batched products).  Automatic: the
    //      smaller estimated time from rates measured on GB300 at o=40
    //      (mixed: triangle 45 TFLOP/s, Alg. 6 products 100, Algs. 4-5
    //      products 35; float64: 0.85 for every operation) plus 10 us per
    //      product launched (it decides at small sizes).
    {
        const double dG = G, dP = P, dO = o, dV = v;
        const double f6_tri = 5.0 * dG * dP * dP * dP;
        const double f6_mm = 2.0 * dG * dP * dP * (dO + dV) + 6.0 * dO * dV * dP * dP +
                             2.0 * dP * dP * dP * dO + 2.0 * dP * dO * dV * dP +
                             (gall_fits ? 0.0 : 2.0 * dG * dP * dP * dO * (nblk6 - 1));
        // per pair (i, j) of Alg. 4 and (j, a) of Alg. 5, products as issued by alg45
        const double p4 = 2.0 * (dV * dV * dP + dV * dG * dV + dG * dG * dV + dO * dG * dG +
                                 dO * dO * dG + dO * dP * dO + dP * dP * dO + dV * dP * dP +
                                 dV * dV * dP + dP * dV * dV + dP * dP * dV);
        const double p5 = 2.0 * (dO * dV * dP + dO * dG * dV + dG * dG * dO + dO * dG * dG +
                                 dO * dV * dG + dV * dP * dO + dP * dP * dV + dO * dP * dP +
                                 dO * dV * dP + dP * dV * dO + dP * dP * dV);
        const double f45 = dO * dO * p4 + dO * dV * p5 + 2.0 * (dO + dV) * dV * dP * dP;
        const bool mixed = !std::is_same<T, double>::value && cfg.tc_products > 0;
        const double n6 = 8.0 * nblk6 + 4.0 * std::ceil(dG / ic) * nblk6;
        const double nb = std::max(1.0, std::min(std::max(dO, dV),
                                                 std::floor(2.0 * (1LL << 30) /
                                                            (dG * dG * sizeof(T)))));
        const double n45 = 13.0 * dO * (std::ceil(dO / nb) + std::ceil(dV / nb)) + 2.0;
        const double t6 = (mixed ? f6_tri / 45e12 + f6_mm / 100e12 : (f6_tri + f6_mm) / 0.85e12) +
                          n6 * 10e-6;
        const double t45 = (mixed ? f45 / 35e12 : f45 / 0.85e12) + n45 * 10e-6;
        t2sq_n5 = cfg.t2sq_route == 2 || (cfg.t2sq_route == 0 && t45 < t6);
    }
    if (!t2sq_n5) {
        gall_resident = gall_fits;
        tri_df = std::is_same<T, double>::value && pol[THC_STEP_TRIANGLE] == THC_POL_FP64_TC;
        tri_pair = std::is_same<T, float>::value && triangle_pair_ok(P);
        if (gall_resident) {
            THC_TRY(Gall.alloc((size_t)G * PP));
            THC_TRY(mm(P, P, o, tr(yo, P), View<T>{U6.p, (long long)G * P, 1}, Gall.p, P, 1, 0,
                       G, 0, P, PP));
            if constexpr (std::is_same<T, double>::value) {
                // The float64-accurate triangle reads G_I^YZ as float pairs.
                if (tri_df)
                    THC_CUDA(split_df(Gall.p, (long long)G * PP,
                                      reinterpret_cast<float2*>(Gall.p), st));
            }
        } else {
            THC_TRY(Gch.alloc((size_t)ic * PP));
        }
        if (tri_df) {
            const size_t pairs = (size_t)ic * ((x6 + 1) / 2) * P;
            THC_TRY(E4.alloc(pairs));
            THC_TRY(F4.alloc(pairs));
        }
        const long long xP = (long long)x6 * P;
        // slabs of C_i, D_a, E and F: an even number of rows for the paired triangle
        const long long xPs = (long long)(tri_pair ? x6 + (x6 & 1) : x6) * P;
        THC_TRY(A6.alloc(ov * P));
        THC_TRY(C6.alloc((size_t)o * xPs));
        THC_TRY(D6.alloc((size_t)v * xPs));
        THC_TRY(Ech.alloc((size_t)ic * xPs));
        THC_TRY(Fch.alloc((size_t)ic * xPs));
        THC_TRY(H.alloc((size_t)x6 * PP));
        THC_TRY(M6.alloc((size_t)x6 * o * P));
        THC_TRY(I6.alloc((size_t)x6 * ov));
    } else {
        // Pairs per batched product: the G x G intermediates of one batch
        // take at most 2 GiB.
        const long long per = (long long)G * G * (long long)sizeof(T);
        nb45 = (int)std::max<long long>(1, std::min<long long>(std::max(o, v), (2LL << 30) / per));
        const long long nb = nb45, mx = std::max(o, v);
        THC_TRY(Q4.alloc(ov * P));
        THC_TRY(S5.alloc(ov * P));
        THC_TRY(C45.alloc((size_t)nb * mx * v));
        THC_TRY(M245.alloc((size_t)nb * mx * G));
        THC_TRY(D45.alloc((size_t)nb * G * G));
        THC_TRY(M345.alloc((size_t)nb * o * G));
        THC_TRY(F45.alloc((size_t)nb * o * mx));
        THC_TRY(M445.alloc((size_t)nb * mx * P));
        THC_TRY(G45.alloc((size_t)nb * PP));
        THC_TRY(M545.alloc((size_t)nb * mx * P));
        THC_TRY(I45.alloc((size_t)nb * mx * v));
        THC_TRY(R45.alloc((size_t)nb * P * v));
    }
    // ---- Alg. 7 scratch; X block: the G x G intermediates take at most
    //      8 GiB (32 X's at most).
    xb = cfg.x_block > 0 ? std::min(cfg.x_block, P)
                         : (int)std::max<long long>(1, std::min<long long>(
                               std::min(P, 32), (8LL << 30) / ((long long)G * G * TB)));
    if (do_alg7) {   // only the shard that evaluates Alg. 7
        THC_TRY(R7.alloc((size_t)P * ov));
        THC_TRY(S7.alloc((size_t)P * ov));
        THC_TRY(C7.alloc((size_t)P * G));
        THC_TRY(D7.alloc((size_t)P * G));
        THC_TRY(Yv.alloc((size_t)xb * o * P));
        THC_TRY(M7.alloc((size_t)xb * o * P));
        THC_TRY(Yo.alloc((size_t)xb * v * P));
        THC_TRY(N7.alloc((size_t)xb * o * G));
        THC_TRY(E7.alloc((size_t)xb * G * G));
        THC_TRY(P7.alloc((size_t)xb * o * G));
        if (!alg7_dense) THC_TRY(G7.alloc((size_t)P * ov));   // G_ia^X for every X
    }
    if (!tcerr.p) THC_TRY(tcerr.alloc(1));
    THC_CUDA(cudaMemsetAsync(tcerr.p, 0, sizeof(int), st));
    // Products of the residual on the routes in use (the tensor-core
    // workspaces are sized from the largest).
    std::vector<Shape> shapes;
    {
        const long long xP = (long long)(tri_pair ? x6 + (x6 & 1) : x6) * P;
        shapes = {
            {P, P, (long long)kb * P, 1}, {(long long)P * kb, P, P, 1}, {P, P, o, kb},
            {P, P, v, kb}, {v, P, v, kb}, {o, G, v, xb}, {G, G, o, xb}, {o, G, G, xb},
            {o, v, G, xb}, {P, P, ov, 1}, {G, P, G, 1}, {P, P, G, 1},
            {P, ov, P, 1}, {o, P, P, xb}, {o, v, P, xb}, {ov, P, P, 1}, {P, P, K, 1}};
        if (alg7_dense) {
            shapes.push_back({P, G, ov, 1});
            shapes.push_back({P, ov, ov, 1});
        }
        if (!t2sq_n5) {
            for (const Shape& sh : std::initializer_list<Shape>{
                     {x6, P, v, o}, {x6, P, o, v}, {ic, xP, o, 1}, {ic, xP, v, 1},
                     {o, P, P, x6}, {o, v, P, x6}, {x6, P, ov, 1}})
                shapes.push_back(sh);
        } else {
            const long long nb = nb45;
            for (const Shape& sh : std::initializer_list<Shape>{
                     {v, v, P, nb}, {v, G, v, nb}, {G, G, v, nb}, {o, G, G, nb},
                     {o, o, G, nb}, {P, P, o, nb}, {v, P, P, nb}, {P, v, v, nb},
                     {P, P, v, nb}, {o, v, P, nb}, {o, G, v, nb}, {G, G, o, nb},
                     {o, v, G, nb}, {v, P, o, nb}, {o, P, P, nb}, {P, v, o, nb},
                     {v, P, P, o}, {o, P, P, v}})
                shapes.push_back(sh);
        }
    }
    bool any_f64tc = cfg.precision == THC_PREC_FP64_TC, any_bf16 = cfg.tc_products > 0;
    for (int st_ = 0; st_ < THC_N_STEPS; ++st_) {
        if (st_ == THC_STEP_TRIANGLE) continue;   // not a product
        any_f64tc = any_f64tc || pol[st_] == THC_POL_FP64_TC;
        any_bf16 = any_bf16 || pol[st_] == THC_POL_BF16X3 || pol[st_] == THC_POL_BF16;
    }
    if (std::is_same<T, double>::value && any_f64tc) {
        // Slices of the largest product's operands and its float64 split-K
        // partials, each at most a quarter of the free memory (a larger
        // product is cut into pieces that fit).
        size_t sl = 0, pt = 0, ex = 0;
        for (const Shape& sh : shapes) {
            size_t a = 0, b = 0, c = 0;
            gemm_f64_tc_sizes((int)std::min<long long>(sh.M, INT32_MAX),
                              (int)std::min<long long>(sh.N, INT32_MAX), (int)sh.K, (int)sh.b,
                              false, &a, &b, &c);
            sl = std::max(sl, a);
            pt = std::max(pt, b);
            ex = std::max(ex, c);
        }
        {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
                pt = std::min(pt, free_b / 4 / sizeof(float));
                sl = std::min(sl, free_b / 4 / sizeof(__nv_bfloat16));
            }
        }
        THC_TRY(f64sl.alloc(sl));
        THC_TRY(f64part.alloc(pt));
        THC_TRY(f64exp.alloc(ex));
        f64ws.slices = f64sl.p;
        f64ws.slice_elems = f64sl.n;
        f64ws.part = f64part.p;
        f64ws.part_elems = f64part.n;
        f64ws.expo = f64exp.p;
        f64ws.expo_elems = f64exp.n;
        f64ws.err = tcerr.p;
        f64tc = true;
    }
    if (std::is_same<T, float>::value && cfg.precision == THC_PREC_MIXED && any_bf16) {
        // Packed-operand workspace: the largest product of the residual.
        size_t need = 0;
        for (const Shape& sh : shapes)
            need = std::max(need, gemm_tc_pack_elems((int)std::min<long long>(sh.M, INT32_MAX),
                                                     (int)std::min<long long>(sh.N, INT32_MAX),
                                                     (int)sh.K, (int)sh.b, false));
        tc_products = cfg.tc_products;
        THC_TRY(tcpack.alloc(need));
        THC_TRY(tcpart.alloc((size_t)std::max<long long>(8 * PP, 1 << 22)));

        tcws.buf = tcpack.p;
        tcws.elems = tcpack.n;
        tcws.partial = tcpart.p;
        tcws.partial_elems = tcpart.n;
        tcws.err = tcerr.p;
        // Buffers that keep their contents for the context's lifetime: their
        // bf16 hi/lo forms are packed once and reused by every residual.
        // The cache may take up to half of the memory left free after init.
        if constexpr (std::is_same<T, float>::value) {
            for (DBuf<T>* b : {&y, &x, &z, &oo, &vv, &S, &KRy, &KRx, &Atil, &U6, &Gall, &Kx})
                if (b->p) pcache.add_constant(b->p, b->n);
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                pcache.budget = std::min<size_t>(free_b / 2, 96ull << 30);
        }
    }
    if (debug_poison()) {
        // NaN bytes in every scratch buffer (not the inputs, the fixed
        // intermediates of init, or the flags that start at zero).
        auto poison = [&](auto& b) -> Err {
            if (b.p) THC_CUDA(cudaMemsetAsync(b.p, 0xff, b.n * sizeof(*b.p), st));
            return Err{};
        };
        for (DBuf<T>* b : {&splitk, &Tc, &t1, &xoo, &xvv, &Ccross, &Abar, &Q, &Wq, &Joo, &Xoo,
                           &Foo, &Jov, &Xov, &Fov, &Jvo, &Xvo, &Fvo, &E1, &Jvv, &Xvv, &Fvv, &ST,
                           &E9, &V9, &O9, &M9, &FvoT, &Lh_oo, &Lh_vv, &Lh_vo, &dtr, &Wfo, &Wfv,
                           &M1, &N1, &M2, &M3, &M4, &M5, &Bbar, &Btil, &C1, &D1, &E, &W, &TA,
                           &Ta0, &D8, &Mo, &A6, &C6, &D6, &Ech, &Fch, &Gch, &H, &M6, &I6, &Q4,
                           &S5, &C45, &M245, &D45, &M345, &F45, &M445, &G45, &M545, &I45, &R45,
                           &W7, &R7, &S7, &C7, &D7, &Yv, &M7, &Yo, &N7, &E7, &P7, &G7, &sigT,
                           &sig1T})
            THC_TRY(poison(*b));
        for (DBuf<double>* b : {&Tcd, &t1d, &sig, &sig1, &en, &red}) THC_TRY(poison(*b));
        THC_TRY(poison(tcpack));
        THC_TRY(poison(tcpart));
        THC_TRY(poison(f64sl));
        THC_TRY(poison(f64part));
        THC_TRY(poison(E4));
        THC_TRY(poison(F4));
    }
    THC_CUDA(cudaStreamSynchronize(st));
    pending = false;
    return Err{};
}

template <typename T>
Err Engine<T>::load(const double* src, T* dst, long long count) {
    if constexpr (std::is_same<T, double>::value) {
        THC_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDefault, st));
    } else {
        DBuf<double> tmp;
        THC_TRY(tmp.alloc(count));
        THC_CUDA(cudaMemcpyAsync(tmp.p, src, sizeof(double) * count, cudaMemcpyDefault, st));
        THC_CUDA(convert(tmp.p, dst, count, st));
        THC_CUDA(cudaStreamSynchronize(st));
    }
    return Err{};
}

template <typename T>
Err Engine<T>::set_state(const double* Zc, const double* t1in) {
    const long long PP = (long long)P * P, ov = (long long)o * v;
    THC_CUDA(cudaMemcpyAsync(Tcd.p, Zc, sizeof(double) * PP, cudaMemcpyDefault, st));
    THC_CUDA(cudaMemcpyAsync(t1d.p, t1in, sizeof(double) * ov, cudaMemcpyDefault, st));
    THC_TRY(check_sym(Tcd.p, P, 1e-12, "Zc"));
    THC_TRY(check_finite(t1d.p, ov, "t1"));
    if constexpr (std::is_same<T, double>::value) {
        THC_CUDA(cudaMemcpyAsync(Tc.p, Tcd.p, sizeof(double) * PP, cudaMemcpyDeviceToDevice, st));
        THC_CUDA(cudaMemcpyAsync(t1.p, t1d.p, sizeof(double) * ov, cudaMemcpyDeviceToDevice, st));
    } else {
        THC_CUDA(convert(Tcd.p, Tc.p, PP, st));
        THC_CUDA(convert(t1d.p, t1.p, ov, st));
    }
    return Err{};
}

template <typename T>
Err Engine<T>::alg6(T* sgm) {
    const long long ov = (long long)o * v, PP = (long long)P * P;
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    seg_begin(THC_STEP_ALG6_GEMM);
    // A_ia^X = sum_Y y_i^Y y_a^Y T^XY  (line 1)
    THC_TRY(mm((int)ov, P, P, rm(KRy.p, P), rm(Tc.p, P), A6.p, P, 1, 0));
    // Blocks of x6 amplitude indices X: every line from 4 on is local to the
    // X rows of C_i, D_a, E, F and H (G_I^YZ is shared by all blocks).
    for (int X0 = x_lo; X0 < x_hi; X0 += x6) {
        const int nX = std::min(x6, x_hi - X0);
        // row slabs of C_i, D_a, E, F: nX rows, or nX rounded up to even
        // with the rows of each pair interleaved for the paired triangle
        const long long xP = (long long)(tri_pair ? nX + (nX & 1) : nX) * P;
        seg_begin(THC_STEP_ALG6_GEMM);
        // C_i^XY (line 4) and D_a^XY (line 5) for the block's X
        THC_TRY(mm(nX, P, v, tr(yv + X0, P), rm(A6.p, P), C6.p, P, 1, 0, o, 0, (long long)v * P,
                   xP));
        THC_TRY(mm(nX, P, o, tr(yo + X0, P), View<T>{A6.p, (long long)v * P, 1}, D6.p, P, 1, 0,
                   v, 0, P, xP));
        if constexpr (std::is_same<T, float>::value) {
            if (tri_pair) {
                // E and F inherit the column order of C_i and D_a (lines 8-9)
                THC_CUDA(pair_rows(C6.p, o, xP, nX, P, st));
                THC_CUDA(pair_rows(D6.p, v, xP, nX, P, st));
            }
        }
        THC_CUDA(cudaMemsetAsync(H.p, 0, sizeof(T) * nX * PP, st));
        for (int I0 = 0; I0 < G; I0 += ic) {
            const int nI = std::min(ic, G - I0);
            seg_begin(THC_STEP_ALG6_GEMM);
            // E^XY = sum_i C_i^XY x_i^I (line 8), F^XZ = sum_a D_a^XZ x_a^I (line 9)
            THC_TRY(mm(nI, (int)xP, o, View<T>{x.p + I0, 1, G}, rm(C6.p, xP), Ech.p, xP, 1, 0));
            THC_TRY(mm(nI, (int)xP, v, View<T>{x.p + (long long)o * G + I0, 1, G}, rm(D6.p, xP),
                       Fch.p, xP, 1, 0));
            const T* Gp;
            if (gall_resident) {
                Gp = Gall.p + (long long)I0 * PP;
            } else {
                THC_TRY(mm(P, P, o, tr(yo, P),
                           View<T>{U6.p + (long long)I0 * P, (long long)G * P, 1}, Gch.p, P, 1,
                           0, nI, 0, P, PP));
                Gp = Gch.p;
            }
            if constexpr (std::is_same<T, double>::value) {
                if (tri_df) {
                    // float pairs of E, F (and of a rebuilt G chunk, in place)
                    THC_CUDA(split_df_pairs(Ech.p, nI, nX, P, E4.p, st));
                    THC_CUDA(split_df_pairs(Fch.p, nI, nX, P, F4.p, st));
                    if (!gall_resident)
                        THC_CUDA(split_df(Gch.p, (long long)nI * PP,
                                          reinterpret_cast<float2*>(Gch.p), st));
                }
            }
            // H^XYZ += (E^XY F^XZ + E^XZ F^XY) G^YZ   (line 11)
            seg_begin(THC_STEP_TRIANGLE);
            // algorithmic count: 5 flops per (I, X, Y, Z)
            if (prof.on) prof.flops[THC_STEP_TRIANGLE] += 5.0 * nI * (double)nX * P * P;
            if constexpr (std::is_same<T, double>::value) {
                if (tri_df)
                    THC_CUDA(triangle_df(H.p, E4.p, F4.p, reinterpret_cast<const float2*>(Gp), P,
                                         nX, nI, st));
                else
                    THC_CUDA(triangle(H.p, Ech.p, Fch.p, Gp, P, nX, nI, st));
            } else if (tri_pair) {
                THC_CUDA(triangle_pair(H.p, reinterpret_cast<const float2*>(Ech.p),
                                       reinterpret_cast<const float2*>(Fch.p), Gp, P, nX, nI, st,
                                       tcerr.p));
            } else {
                THC_CUDA(triangle(H.p, Ech.p, Fch.p, Gp, P, nX, nI, st));
            }
            seg_end();
        }
        seg_begin(THC_STEP_ALG6_POST);
        // I_ia = sum_YZ y_i^Z y_a^Y H^XYZ (line 14); sigma^XX' += sum_ia y_i^X' y_a^X' I_ia
        THC_TRY(mm(o, P, P, rm(yo, P), View<T>{H.p, 1, P}, M6.p, P, 1, 0, nX, 0, PP,
                   (long long)o * P));
        THC_TRY(mm(o, v, P, rm(M6.p, P), tr(yv, P), I6.p, v, 1, 0, nX, (long long)o * P, 0, ov));
        THC_TRY(mm(nX, P, (int)ov, rm(I6.p, ov), rm(KRy.p, P), sgm + (long long)X0 * P, P, 1, 1));
    }
    return Err{};
}

// Algs. 4 and 5: the T2^2 contributions to Omega^A (Eq. 32) and Omega^C
// (Eq. 33) through per-pair two-index products, O(o^2 v G^2).  With the
// Khatri-Rao rows W_i[a][Z] = y_i^Z y_a^Z (= U_a[i][Z]):
//   Alg. 4, pair (i, j):  C = (W_i T) W_j^T = t_ij^cd,  D = x_v^T C x_v,
//     E = z o D,  F = x_o E x_o^T = sum_cd t_ij^cd (kc|ld),
//     H = T o (y_o^T F y_o),  I = y_v H y_v^T = sigma_ij^ab,
//     sigma^XX' += sum_ab W_i[a][X] I_ab W_j[b][X'];
//   Alg. 5, pair (j, a):  C = (U_a T) W_j^T = t_lj^ad,  D = x_o^T C x_v,
//     E = z o D,  F = x_o E^T x_v^T = sum_ld t_lj^ad (lc|kd),
//     H = T o (y_v^T F^T y_o),  I = y_o H y_v^T,
//     sigma^XX' += sum_ib U_a[i][X] I_ib W_j[b][X'].
// Each loop runs over one index with the other batched (nb45 pairs a launch).
template <typename T>
Err Engine<T>::alg45(T* sgm) {
    const long long ov = (long long)o * v, PP = (long long)P * P, GG = (long long)G * G;
    const long long vP = (long long)v * P, oP = (long long)o * P;
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    const T* xo = x.p;
    const T* xv = x.p + (long long)o * G;
    const T* kr = KRy.p;
    seg_begin(THC_STEP_ALG6_GEMM);
    // Q_i = W_i T (v x P, for every i);  S_a = U_a T (o x P, for every a)
    THC_TRY(mm(v, P, P, rm(kr, P), rm(Tc.p, P), Q4.p, P, 1, 0, o, vP, 0, vP));
    THC_TRY(mm(o, P, P, View<T>{kr, vP, 1}, rm(Tc.p, P), S5.p, P, 1, 0, v, P, 0, oP));
    // ---- Alg. 4: loop over i, batch over j
    for (int i = 0; i < o; ++i) {
        for (int j0 = 0; j0 < o; j0 += nb45) {
            const int nb = std::min(nb45, o - j0);
            const T* Wj = kr + (long long)j0 * vP;
            THC_TRY(mm(v, v, P, rm(Q4.p + (long long)i * vP, P), tr(Wj, P), C45.p, v, 1, 0, nb,
                       0, vP, (long long)v * v));
            THC_TRY(mm(v, G, v, rm(C45.p, v), rm(xv, G), M245.p, G, 1, 0, nb, (long long)v * v, 0,
                       (long long)v * G));
            THC_TRY(mm(G, G, v, tr(xv, G), rm(M245.p, G), D45.p, G, 1, 0, nb, 0,
                       (long long)v * G, GG));
            THC_CUDA(hadamard_batched(D45.p, z.p, GG, nb, st));
            THC_TRY(mm(o, G, G, rm(xo, G), rm(D45.p, G), M345.p, G, 1, 0, nb, 0, GG,
                       (long long)o * G));
            THC_TRY(mm(o, o, G, rm(M345.p, G), tr(xo, G), F45.p, o, 1, 0, nb, (long long)o * G, 0,
                       (long long)o * o));
            THC_TRY(mm(o, P, o, rm(F45.p, o), rm(yo, P), M445.p, P, 1, 0, nb, (long long)o * o, 0,
                       oP));
            THC_TRY(mm(P, P, o, tr(yo, P), rm(M445.p, P), G45.p, P, 1, 0, nb, 0, oP, PP));
            THC_CUDA(hadamard_batched(G45.p, Tc.p, PP, nb, st));
            THC_TRY(mm(v, P, P, rm(yv, P), rm(G45.p, P), M545.p, P, 1, 0, nb, 0, PP, vP));
            THC_TRY(mm(v, v, P, rm(M545.p, P), tr(yv, P), I45.p, v, 1, 0, nb, vP, 0,
                       (long long)v * v));
            THC_TRY(mm(P, v, v, tr(kr + (long long)i * vP, P), rm(I45.p, v), R45.p, v, 1, 0, nb,
                       0, (long long)v * v, vP));
            THC_TRY(mm(P, P, v, rm(R45.p, v), rm(Wj, P), sgm, P, 1, 1, nb, vP, vP, 0, true));
        }
    }
    // ---- Alg. 5: loop over j, batch over a
    for (int j = 0; j < o; ++j) {
        const T* Wj = kr + (long long)j * vP;
        for (int a0 = 0; a0 < v; a0 += nb45) {
            const int nb = std::min(nb45, v - a0);
            THC_TRY(mm(o, v, P, rm(S5.p + (long long)a0 * oP, P), tr(Wj, P), C45.p, v, 1, 0, nb,
                       oP, 0, ov));
            THC_TRY(mm(o, G, v, rm(C45.p, v), rm(xv, G), M245.p, G, 1, 0, nb, ov, 0,
                       (long long)o * G));
            THC_TRY(mm(G, G, o, tr(xo, G), rm(M245.p, G), D45.p, G, 1, 0, nb, 0,
                       (long long)o * G, GG));
            THC_CUDA(hadamard_batched(D45.p, z.p, GG, nb, st));
            THC_TRY(mm(o, G, G, rm(xo, G), tr(D45.p, G), M345.p, G, 1, 0, nb, 0, GG,
                       (long long)o * G));
            THC_TRY(mm(o, v, G, rm(M345.p, G), tr(xv, G), F45.p, v, 1, 0, nb, (long long)o * G, 0,
                       ov));
            THC_TRY(mm(v, P, o, tr(F45.p, v), rm(yo, P), M445.p, P, 1, 0, nb, ov, 0, vP));
            THC_TRY(mm(P, P, v, tr(yv, P), rm(M445.p, P), G45.p, P, 1, 0, nb, 0, vP, PP));
            THC_CUDA(hadamard_batched(G45.p, Tc.p, PP, nb, st));
            THC_TRY(mm(o, P, P, rm(yo, P), rm(G45.p, P), M545.p, P, 1, 0, nb, 0, PP, oP));
            THC_TRY(mm(o, v, P, rm(M545.p, P), tr(yv, P), I45.p, v, 1, 0, nb, oP, 0, ov));
            THC_TRY(mm(P, v, o, View<T>{kr + (long long)a0 * P, 1, vP}, rm(I45.p, v), R45.p, v, 1,
                       0, nb, P, ov, vP));
            THC_TRY(mm(P, P, v, rm(R45.p, v), rm(Wj, P), sgm, P, 1, 1, nb, vP, 0, 0, true));
        }
    }
    return Err{};
}

template <typename T>
Err Engine<T>::alg7(T* sgm) {
    const long long ov = (long long)o * v, PP = (long long)P * P, GG = (long long)G * G;
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    const T* xo = x.p;
    const T* xv = x.p + (long long)o * G;
    seg_begin(THC_STEP_ALG7);
    // R_ia^X = 2 sum_Y y_i^Y y_a^Y (S T)^XY + S_ia^X   (lines 3-8)
    THC_TRY(mm(P, (int)ov, P, rm(ST.p, P), tr(KRy.p, P), R7.p, ov, 2, 0));
    for (int X0 = 0; X0 < P; X0 += xb) {
        const int nx = std::min(xb, P - X0);
        THC_CUDA(scale_rows(yo, o, P, vv.p, X0, nx, Yv.p, st));
        THC_TRY(mm(o, P, P, rm(Yv.p, P), rm(Tc.p, P), M7.p, P, 1, 0, nx, (long long)o * P, 0,
                   (long long)o * P));
        THC_CUDA(scale_rows(yv, v, P, oo.p, X0, nx, Yo.p, st));
        THC_TRY(mm(o, v, P, rm(M7.p, P), View<T>{Yo.p, 1, P}, S7.p + (long long)X0 * ov, v, -1,
                   0, nx, (long long)o * P, (long long)v * P, ov));
    }
    THC_CUDA(lincomb(R7.p, (long long)P * ov, 1, R7.p, 1, S7.p, 0, (const T*)nullptr, st));
    if (alg7_dense) {
        // Coulomb part: C^XI = sum_ia x_i^I x_a^I R_ia^X, D = C z (lines 9-10)
        THC_TRY(mm(P, G, (int)ov, rm(R7.p, ov), rm(KRx.p, G), C7.p, G, 1, 0));
        THC_TRY(mm(P, G, G, rm(C7.p, G), rm(z.p, G), D7.p, G, 1, 0));
        THC_TRY(mm(P, P, G, rm(C7.p, G), tr(D7.p, G), sgm, P, 1, 1));
        // Exchange parts through the dense (ib|ja): sigma -= 1/2 R Kx R^T,
        // sigma += 1/2 S Kx S^T (the same sums as lines 12-22).
        for (int pass = 0; pass < 2; ++pass) {
            const T* src = pass == 0 ? R7.p : S7.p;
            const double sign = pass == 0 ? -0.5 : 0.5;
            THC_TRY(mm(P, (int)ov, (int)ov, rm(src, ov), rm(Kx.p, ov), W7.p, ov, 1, 0));
            THC_TRY(mm(P, P, (int)ov, rm(W7.p, ov), tr(src, ov), sgm, P, sign, 1));
        }
        return Err{};
    }
    // Exchange parts (lines 12-21), blocked over X
    for (int pass = 0; pass < 2; ++pass) {
        const T* src = pass == 0 ? R7.p : S7.p;
        const double sign = pass == 0 ? -0.5 : 0.5;
        for (int X0 = 0; X0 < P; X0 += xb) {
            const int nx = std::min(xb, P - X0);
            THC_TRY(mm(o, G, v, rm(src + (long long)X0 * ov, v), rm(xv, G), N7.p, G, 1, 0, nx,
                       ov, 0, (long long)o * G));
            // Coulomb part (line 9) from the same product: C^XI = sum_i x_i^I
            // (R_X x_v)_i^I, stored transposed (C7[I][X])
            if (pass == 0) THC_CUDA(diag_reduce(xo, N7.p, o, G, nx, C7.p, P, X0, st));
            THC_TRY(mm(G, G, o, tr(xo, G), rm(N7.p, G), E7.p, G, 1, 0, nx, 0, (long long)o * G,
                       GG));
            THC_CUDA(hadamard_batched(E7.p, z.p, GG, nx, st));
            THC_TRY(mm(o, G, G, rm(xo, G), tr(E7.p, G), P7.p, G, 1, 0, nx, 0, GG,
                       (long long)o * G));
            THC_TRY(mm(o, v, G, rm(P7.p, G), tr(xv, G), G7.p + (long long)X0 * ov, v, 1, 0, nx,
                       (long long)o * G, 0, ov));
        }
        // sigma^XX' += sign sum_ia G_ia^X src_ia^X' for all X at once, so
        // that src is packed for the tensor cores once per pass.
        THC_TRY(mm(P, P, (int)ov, rm(G7.p, ov), tr(src, ov), sgm, P, sign, 1));
    }
    // D^T = z C^T (line 10, z symmetric); sigma += C D^T
    THC_TRY(mm(G, P, G, rm(z.p, G), rm(C7.p, P), D7.p, P, 1, 0));
    THC_TRY(mm(P, P, G, tr(C7.p, P), rm(D7.p, P), sgm, P, 1, 1));
    return Err{};
}

template <typename T>
Err Engine<T>::residual_dev(bool want_energy) {
    const long long ov = (long long)o * v, PP = (long long)P * P;
    const long long oo2 = (long long)o * o, vv2 = (long long)v * v;
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    T* sgm;
    T* sg1;
    if constexpr (std::is_same<T, double>::value) {
        sgm = sig.p;
        sg1 = sig1.p;
    } else {
        sgm = sigT.p;
        sg1 = sig1T.p;
    }
    THC_CUDA(cudaMemsetAsync(sgm, 0, sizeof(T) * PP, st));
    THC_CUDA(cudaMemsetAsync(sg1, 0, sizeof(T) * ov, st));
    for (DBuf<T>* b : {&xoo, &xvv, &Ccross, &Joo, &Jov, &Jvo, &Jvv, &Xoo, &Xov, &Xvo, &Xvv})
        THC_CUDA(cudaMemsetAsync(b->p, 0, b->n * sizeof(T), st));

    // ---- fused Cholesky-slab pass: Algs. 1, 2, 3, 8 and the Fock matrix
    for (int A0 = 0; A0 < K; A0 += kb) {
        const int nb = std::min(kb, K - A0);
        const T* Lov_s = Lov.p + A0 * ov;
        seg_begin(THC_STEP_DRESS);
        THC_TRY(dress(Loo.p + A0 * oo2, Lov_s, Lvv.p + A0 * ((long long)v * (v + 1) / 2), nb,
                      Lh_oo.p, Lh_vv.p, Lh_vo.p));
        seg_begin(THC_STEP_FOCK);
        THC_TRY(fock_slab(nb, Lh_oo.p, Lov_s, Lh_vo.p, Lh_vv.p));
        seg_begin(THC_STEP_ALG1);
        // Alg. 1: Bbar^XY = sum_ik y_i^X l_ki y_k^Y, Btil^XY = sum_ac y_a^X l_ac y_c^Y,
        // C = v o Bbar - o o Btil, sigma += C T C^T.  Alg. 3: Ccross += Bbar o Btil.
        THC_TRY(mm(o, P, o, rm(Lh_oo.p, o), rm(yo, P), M1.p, P, 1, 0, nb, oo2, 0, (long long)o * P));
        THC_TRY(mm(P, P, o, tr(M1.p, P), rm(yo, P), Bbar.p, P, 1, 0, nb, (long long)o * P, 0, PP));
        THC_TRY(mm(v, P, v, rm(Lh_vv.p, v), rm(yv, P), N1.p, P, 1, 0, nb, vv2, 0, (long long)v * P));
        THC_TRY(mm(P, P, v, tr(yv, P), rm(N1.p, P), Btil.p, P, 1, 0, nb, 0, (long long)v * P, PP));
        THC_CUDA(alg1_combine(Bbar.p, Btil.p, oo.p, vv.p, C1.p, Ccross.p, P, nb, st));
        THC_TRY(mm(P * nb, P, P, rm(C1.p, P), rm(Tc.p, P), D1.p, P, 1, 0));
        THC_TRY(mm(P, P, nb * P, rm(D1.p, (long long)nb * P), tr(C1.p, (long long)nb * P), sgm,
                   P, 1, 1));
        seg_begin(THC_STEP_ALG2_8);
        // Alg. 2 line 5: Abar^X = sum_ai y_a^X y_i^X l_ai
        THC_TRY(mm(v, P, o, rm(Lh_vo.p, o), rm(yo, P), M2.p, P, 1, 0, nb, ov, 0, (long long)v * P));
        THC_CUDA(diag_reduce(yv, M2.p, v, P, nb, Abar.p, K, A0, st));
        // Alg. 8 lines 6-9: D_ia = sum_kc u_ik^ac l_kc; Alg. 2: Q^X = (2 Dtil - H)^X
        THC_TRY(d_operator(Lov_s, nb, D8.p));
        THC_TRY(mm(o, P, v, rm(D8.p, v), rm(yv, P), M5.p, P, 1, 0, nb, ov, 0, (long long)o * P));
        THC_CUDA(diag_reduce(yo, M5.p, o, P, nb, Q.p, K, A0, st));
        // Alg. 8 lines 10-13
        THC_TRY(mm(o, o, v, rm(Lov_s, v), tr(D8.p, v), xoo.p, o, 1, 1, nb, ov, ov, 0, true));
        THC_TRY(mm(v, v, o, tr(D8.p, v), rm(Lov_s, v), xvv.p, v, -1, 1, nb, ov, ov, 0, true));
        THC_TRY(mm(o, v, v, rm(D8.p, v), tr(Lh_vv.p, v), sg1, v, 1, 1, nb, ov, vv2, 0, true));
        THC_TRY(mm(o, v, o, tr(Lh_oo.p, o), rm(D8.p, v), sg1, v, -1, 1, nb, oo2, ov, 0, true));
    }

    seg_begin(THC_STEP_POST);
    // Alg. 2 line 14: sigma += Abar Abar^T + Q Abar^T + Abar Q^T
    THC_CUDA(lincomb(Wq.p, (long long)P * K, 1, Abar.p, 1, Q.p, 0, (const T*)nullptr, st));
    THC_TRY(mm(P, P, K, rm(Wq.p, K), tr(Abar.p, K), sgm, P, 1, 1));
    THC_TRY(mm(P, P, K, rm(Abar.p, K), tr(Q.p, K), sgm, P, 1, 1));
    // Alg. 3 lines 11-12: sigma -= (S T) Ccross^T + Ccross (S T)^T
    THC_TRY(mm(P, P, P, rm(S.p, P), rm(Tc.p, P), ST.p, P, 1, 0));
    THC_TRY(mm(P, P, P, rm(ST.p, P), tr(Ccross.p, P), sgm, P, -1, 1));
    THC_TRY(mm(P, P, P, rm(Ccross.p, P), tr(ST.p, P), sgm, P, -1, 1));

    // Dressed Fock matrix  F^ = dress(f) + 2 J - X  (see fock_slab)
    // (on a sharded context the orbital-energy terms dress(f) belong to the
    // first shard; J and X are the shard's partial sums over its vectors)
    const double fw = f_terms ? 1.0 : 0.0;
    THC_CUDA(eps_t1(epsT.p, t1.p, o, v, E1.p, st));
    THC_CUDA(lincomb(Foo.p, oo2, fw, foo.p, 2, Joo.p, -1, Xoo.p, st));
    THC_CUDA(lincomb(Fov.p, ov, 2, Jov.p, -1, Xov.p, 0, (const T*)nullptr, st));
    THC_CUDA(lincomb(Fvo.p, ov, fw, E1.p, 2, Jvo.p, -1, Xvo.p, st));
    THC_CUDA(lincomb(Fvv.p, vv2, fw, fvv.p, 2, Jvv.p, -1, Xvv.p, st));

    // Alg. 9: E = o o (y_v^T Fb_vv y_v) - v o (y_o^T Fb_oo^T y_o), sigma += E B^T + B E^T
    THC_CUDA(lincomb(xoo.p, oo2, 1, Foo.p, 1, xoo.p, 0, (const T*)nullptr, st));
    THC_CUDA(lincomb(xvv.p, vv2, 1, Fvv.p, 1, xvv.p, 0, (const T*)nullptr, st));
    THC_TRY(mm(v, P, v, rm(xvv.p, v), rm(yv, P), M9.p, P, 1, 0));
    THC_TRY(mm(P, P, v, tr(yv, P), rm(M9.p, P), V9.p, P, 1, 0));
    THC_TRY(mm(o, P, o, tr(xoo.p, o), rm(yo, P), M9.p, P, 1, 0));
    THC_TRY(mm(P, P, o, tr(yo, P), rm(M9.p, P), O9.p, P, 1, 0));
    THC_CUDA(hadamard2(E9.p, PP, oo.p, V9.p, vv.p, O9.p, st));
    THC_TRY(mm(P, P, P, rm(E9.p, P), tr(ST.p, P), sgm, P, 1, 1));
    THC_TRY(mm(P, P, P, rm(ST.p, P), tr(E9.p, P), sgm, P, 1, 1));

    // Alg. 10: sigma_ia += F^_ai + sum_kc u_ik^ac F^_kc
    THC_TRY(d_operator(Fov.p, 1, D8.p));
    THC_CUDA(transpose_batched(Fvo.p, FvoT.p, 1, v, o, st));
    THC_CUDA(lincomb(sg1, ov, 1, sg1, 1, D8.p, 1, FvoT.p, st));

    // Algs. 6 and 7 (T2^2 terms through the THC ovov integrals)
    if (t2sq_n5) {
        if (ish == 0) THC_TRY(alg45(sgm));
    } else {
        THC_TRY(alg6(sgm));
    }
    if (do_alg7) THC_TRY(alg7(sgm));

    seg_begin(THC_STEP_POST);
    if constexpr (!std::is_same<T, double>::value) {
        THC_CUDA(cudaMemsetAsync(sig.p, 0, sizeof(double) * PP, st));
        THC_CUDA(cudaMemsetAsync(sig1.p, 0, sizeof(double) * ov, st));
        THC_CUDA(accumulate(sig.p, sgm, PP, 1.0, st));
        THC_CUDA(accumulate(sig1.p, sg1, ov, 1.0, st));
    }
    if (want_energy) THC_TRY(energy_dev());
    seg_end();
    return Err{};
}

template <typename T>
Err Engine<T>::energy_dev() {
    const long long PP = (long long)P * P, ov = (long long)o * v, oo2 = (long long)o * o;
    // doubles: <Zc, Wen>;  singles: sum_A [2 (L_A . t1)^2 - tr((L_A t1^T)^2)]
    seg_begin(THC_STEP_ENERGY);
    THC_CUDA(dot(Tcd.p, Wen.p, PP, red.p, en.p, st));
    THC_TRY(mm(o, o, v, rm(Lov.p, v), tr(t1.p, v), Mo.p, o, 1, 0, K, ov, 0, oo2));
    THC_CUDA(singles_energy(Lov.p, Mo.p, t1.p, K, o, v, red.p, en.p + 1, st));
    return Err{};
}

template <typename T>
Err Engine<T>::residual(const double* Zc, const double* t1in, double* sigmaZ,
                        double* sigma1, double* energy_out) {
    THC_TRY(set_state(Zc, t1in));
    THC_TRY(residual_dev(energy_out != nullptr));
    THC_TRY(prof_collect());
    THC_TRY(check_timeout());
    const long long PP = (long long)P * P, ov = (long long)o * v;
    THC_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    THC_CUDA(any_nonfinite(sig.p, PP, flag.p, st));
    THC_CUDA(any_nonfinite(sig1.p, ov, flag.p, st));
    THC_CUDA(cudaMemcpyAsync(sigmaZ, sig.p, sizeof(double) * PP, cudaMemcpyDefault, st));
    THC_CUDA(cudaMemcpyAsync(sigma1, sig1.p, sizeof(double) * ov, cudaMemcpyDefault, st));
    int bad = 0;
    double e[2] = {0, 0};
    THC_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (energy_out) THC_CUDA(cudaMemcpyAsync(e, en.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    THC_CUDA(cudaStreamSynchronize(st));
    if (energy_out) {
        const double etot = e[0] + e[1];
        THC_CUDA(cudaMemcpy(energy_out, &etot, sizeof(double), cudaMemcpyDefault));
    }
    if (bad) return Err{THC_ERR_NUMERIC, "residual has non-finite entries"};
    return Err{};
}

template <typename T>
Err Engine<T>::energy(const double* Zc, const double* t1in, double* e_out) {
    THC_TRY(set_state(Zc, t1in));
    THC_TRY(energy_dev());
    double e[2];
    THC_CUDA(cudaMemcpyAsync(e, en.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    THC_CUDA(cudaStreamSynchronize(st));
    const double etot = e[0] + e[1];
    THC_CUDA(cudaMemcpy(e_out, &etot, sizeof(double), cudaMemcpyDefault));
    return Err{};
}

// App. II: D_ij = -2 sum_kab t_ik^ab (2 t_jk^ab - t_jk^ba) and
// D_ab = 2 sum_ijc t_ij^ac (2 t_ij^bc - t_ji^bc) (Eqs. 47-48) for the THC
// amplitudes t = y y T y y, in O(N^4) with o = y_o^T y_o, v = y_v^T y_v:
//   Coulomb (Eqs. 53-54):  M = T (o o v) T,
//     D_oo = -4 y_o (v o M) y_o^T,   D_vv = 4 y_v (o o M) y_v^T;
//   exchange (Eqs. 55-56), per occupied i (virtual a) with A = T diag(y_i) v
//   (T diag(y_a) o):  B = (o o A) T^T (resp. (v o A) T^T),
//     c[Y] = sum_X v^XY B^XY (resp. o^XY B^XY),
//     D_ij += 2 sum_Y c_i[Y] y_j^Y,   D_ab -= 2 sum_Y c_a[Y] y_b^Y.
template <typename T>
Err Engine<T>::mp2_density(const double* Zc, double* Doo_out, double* Dvv_out) {
    const long long PP = (long long)P * P;
    const T* yo = y.p;
    const T* yv = y.p + (long long)o * P;
    const int mx = std::max(o, v);
    if (!dn_ones.p) {
        const long long per = 2 * PP * (long long)sizeof(T);
        const int nb = (int)std::max<long long>(1, std::min<long long>(mx, (2LL << 30) / per));
        THC_TRY(dn_x1.alloc((size_t)nb * PP));
        THC_TRY(dn_x2.alloc((size_t)nb * PP));
        THC_TRY(dn_c.alloc((size_t)nb * P));
        THC_TRY(dn_m1.alloc(PP));
        THC_TRY(dn_m2.alloc(PP));
        THC_TRY(dn_q.alloc((size_t)mx * P));
        THC_TRY(dn_oo.alloc((size_t)o * o));
        THC_TRY(dn_vv.alloc((size_t)v * v));
        THC_TRY(dn_t1.alloc((size_t)o * v));
        THC_TRY(dn_out.alloc((size_t)o * o + (size_t)v * v));
        THC_TRY(dn_ones.alloc(P));
        std::vector<T> one(P, T(1));
        THC_CUDA(cudaMemcpyAsync(dn_ones.p, one.data(), sizeof(T) * P, cudaMemcpyHostToDevice, st));
        THC_CUDA(cudaMemsetAsync(dn_t1.p, 0, sizeof(T) * o * v, st));
    }
    const int nbmax = (int)(dn_c.n / P);
    // the core (t1 = 0 here; the singles play no part in Eqs. 47-48)
    std::vector<double> zero((size_t)o * v, 0.0);
    THC_TRY(set_state(Zc, zero.data()));
    // Coulomb parts
    THC_TRY(mm(P, P, P, rm(Tc.p, P), rm(S.p, P), dn_m1.p, P, 1, 0));
    THC_TRY(mm(P, P, P, rm(dn_m1.p, P), rm(Tc.p, P), dn_m2.p, P, 1, 0));
    THC_CUDA(hadamard2(dn_m1.p, PP, vv.p, dn_m2.p, (const T*)nullptr, (const T*)nullptr, st));
    THC_TRY(mm(o, P, P, rm(yo, P), rm(dn_m1.p, P), dn_q.p, P, 1, 0));
    THC_TRY(mm(o, o, P, rm(dn_q.p, P), tr(yo, P), dn_oo.p, o, -4, 0));
    THC_CUDA(hadamard2(dn_m1.p, PP, oo.p, dn_m2.p, (const T*)nullptr, (const T*)nullptr, st));
    THC_TRY(mm(v, P, P, rm(yv, P), rm(dn_m1.p, P), dn_q.p, P, 1, 0));
    THC_TRY(mm(v, v, P, rm(dn_q.p, P), tr(yv, P), dn_vv.p, v, 4, 0));
    // exchange parts: pass 0 over occupied i, pass 1 over virtual a
    for (int pass = 0; pass < 2; ++pass) {
        const int R = pass == 0 ? o : v;
        const T* yr = pass == 0 ? yo : yv;
        const T* inner = pass == 0 ? vv.p : oo.p;    // A = T diag(y_r) inner
        const T* mask = pass == 0 ? oo.p : vv.p;     // B = (mask o A) T^T
        const T* wsum = pass == 0 ? vv.p : oo.p;     // c = sum_X wsum^XY B^XY
        T* D = pass == 0 ? dn_oo.p : dn_vv.p;
        const double sign = pass == 0 ? 2.0 : -2.0;
        for (int r0 = 0; r0 < R; r0 += nbmax) {
            const int nb = std::min(nbmax, R - r0);
            // x1[b] = T diag(y_r0+b): T[W][X] y^X  (T symmetric, so this is T^T diag(y))
            THC_CUDA(scale_rows(Tc.p, P, P, yr, r0, nb, dn_x1.p, st));
            THC_TRY(mm(P, P, P, rm(dn_x1.p, P), rm(inner, P), dn_x2.p, P, 1, 0, nb, PP, 0, PP));
            THC_CUDA(hadamard_batched(dn_x2.p, mask, PP, nb, st));
            THC_TRY(mm(P, P, P, rm(dn_x2.p, P), tr(Tc.p, P), dn_x1.p, P, 1, 0, nb, PP, 0, PP));
            THC_CUDA(hadamard_batched(dn_x1.p, wsum, PP, nb, st));
            THC_TRY(mm(1, P, P, View<T>{dn_ones.p, 0, 1}, rm(dn_x1.p, P), dn_c.p, P, 1, 0, nb, 0,
                       PP, P));
            THC_TRY(mm(nb, R, P, rm(dn_c.p, P), tr(yr, P), D + (long long)r0 * R, R, sign, 1));
        }
    }
    THC_CUDA(to_double(dn_oo.p, dn_out.p, (long long)o * o, st));
    THC_CUDA(to_double(dn_vv.p, dn_out.p + (long long)o * o, (long long)v * v, st));
    THC_CUDA(cudaMemcpyAsync(Doo_out, dn_out.p, sizeof(double) * o * o, cudaMemcpyDefault, st));
    THC_CUDA(cudaMemcpyAsync(Dvv_out, dn_out.p + (long long)o * o, sizeof(double) * v * v,
                             cudaMemcpyDefault, st));
    THC_CUDA(cudaStreamSynchronize(st));
    return Err{};
}

template struct Engine<double>;
template struct Engine<float>;

}  // namespace thc
