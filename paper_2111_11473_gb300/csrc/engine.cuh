// Residual engine of the THC-RR-CCSD library: device buffers and the
// factorised evaluation of Algorithms 1-10.
#pragma once

#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "kernels.cuh"

namespace thc {

// Owned device allocation.
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    Err alloc(size_t count) {
        n = count;
        if (count == 0) return Err{};
        if (debug_alloc_fails()) {
            n = 0;
            return Err{THC_ERR_OOM, "device allocation failed (injected by THC_FAIL_ALLOC_AT)"};
        }
        const cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();   // a failed allocation must not surface at a later check
            p = nullptr;
            n = 0;
            return Err{e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA,
                       "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                           " bytes: " + cudaGetErrorString(e)};
        }
        return Err{};
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DBuf() { if (p) cudaFree(p); }
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
};

long long launches();

// Per-step device timing with CUDA events on the engine's stream.
struct Profiler {
    bool on = false;
    int cur = -1;
    double ms[THC_N_STEPS] = {};
    double flops[THC_N_STEPS] = {};
    long long launches[THC_N_STEPS] = {};
    long long residuals = 0;
    long long launch_base = 0, kernel_launches = 0;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<int, int>>> marks;   // (step, (ev0, ev1))
    int used = 0;
    cudaEvent_t next_event() {
        if (used == (int)pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void reset() {
        for (int i = 0; i < THC_N_STEPS; ++i) ms[i] = flops[i] = 0, launches[i] = 0;
        residuals = 0;
        launch_base = thc::launches();
        kernel_launches = 0;
    }
    ~Profiler() { for (auto e : pool) cudaEventDestroy(e); }
};

// Matrix-product policy: which kernel family runs the contractions.
enum class MMKind { SIMT, TC_BF16X3 };

template <typename T>
struct Engine {
    int o = 0, v = 0, n = 0, P = 0, G = 0, K = 0;
    // Shard of a multi-GPU split: Cholesky vectors [K0, K0 + K) of Kglob
    // (K is the local count), Alg. 6 rows [x_lo, x_hi), Alg. 7 and the
    // orbital-energy Fock terms on one shard each.
    int Kglob = 0, K0 = 0, x_lo = 0, x_hi = 0, nsh = 1, ish = 0;
    bool do_alg7 = true, f_terms = true;
    int kb = 0, ic = 0, xb = 0;
    int x6 = 0;                             // amplitude indices X per Alg. 6 block
    bool gall_resident = false;
    MMKind mm_kind = MMKind::SIMT;
    cudaStream_t st = nullptr;
    size_t bytes = 0;
    Profiler prof;
    bool nvtx_open = false;                 // an NVTX step range is open
    int step_now = -1;                      // step being evaluated (THC_STEP_*), -1 outside
    int pol[THC_N_STEPS] = {};              // resolved per-step arithmetic (THC_POL_*)
    bool f64tc_default = false;             // context policy outside the steps
    // Tensor-core products per contraction of the current step (float engine).
    int step_tcp() const {
        if (step_now < 0) return tc_products;
        const int p = pol[step_now];
        return p == THC_POL_BF16X3 ? 3 : (p == THC_POL_BF16 ? 1 : 0);
    }
    // Float64 products of the current step on the tensor cores.
    bool step_f64tc() const {
        return f64tc && (step_now < 0 ? f64tc_default : pol[step_now] == THC_POL_FP64_TC);
    }
    // Open / close a timed segment of step `step` (no-ops when profiling is off).
    void seg_begin(int step);
    void seg_end();
    void prof_close();                      // close the open timed segment
    Err prof_collect();

    // Fixed data (storage type T unless noted).
    DBuf<T> y, x, z;                        // n x P, n x G, G x G
    DBuf<T> Loo, Lov, Lvv;                  // K x o x o, K x o x v, K x v(v+1)/2 (undressed;
                                            // Lvv holds lower triangles, row a: b <= a)
    DBuf<T> foo, fvv;                       // diagonal Fock blocks diag(eps_o), diag(eps_v)
    DBuf<T> epsT;                           // n orbital energies
    DBuf<T> oo, vv, S;                      // P x P
    DBuf<T> KRy, KRx;                       // (o v) x P, (o v) x G (KRx: dense Alg. 7 only)
    DBuf<T> Atil;                           // P x K   (Alg. 2 line 6 / Alg. 8 line 6)
    DBuf<double> Wen;                       // P x P   energy weight of the core
    DBuf<T> Gall;                           // G x P x P (Alg. 6 line 10), if resident
    DBuf<T> B6;                             // (o v) x G (Alg. 6 line 2), init only
    DBuf<T> U6;                             // o x G x P  sum_a B_ia^I y_a^Z

    // Per-residual state and accumulators.
    DBuf<T> Tc, t1;                         // P x P, o x v
    DBuf<double> Tcd, t1d;                  // float64 copies of the state
    DBuf<double> sig, sig1, en;             // P x P, o x v, energy scalars
    DBuf<T> sigT, sig1T;                    // partial sums in T (float engine)
    DBuf<T> splitk;                         // split-K partials of the GEMMs
    int tc_products = 0;                    // tensor-core products (float engine)
    DBuf<__nv_bfloat16> tcpack;             // packed bf16 hi/lo operands
    DBuf<float> tcpart;                     // tensor-core split-K partials
    DBuf<int> tcerr;                        // bounded-wait expiry flag
    TcWorkspace tcws;
    PackCache pcache;                       // packed constant operands (float engine)
    bool f64tc = false;                     // float64 products on the tensor cores
    F64TcWorkspace f64ws;
    DBuf<__nv_bfloat16> f64sl;              // operand slices
    DBuf<float> f64part;                    // slice-pair products
    DBuf<int> f64exp;                       // per-row exponents
    ~Engine() { pcache.release(); }
    Err check_timeout();
    std::vector<double> eps_h;              // orbital energies (host copy)
    DBuf<T> xoo, xvv, Ccross, Abar, Q;      // o x o, v x v, P x P, P x K, P x K
    DBuf<T> Joo, Jov, Jvo, Jvv, Xoo, Xov, Xvo, Xvv;  // t1 parts of the Fock matrix
    DBuf<T> Foo, Fov, Fvo, Fvv;             // dressed Fock blocks
    DBuf<T> E1;                             // v x o: (eps_a - eps_i) t_i^a
    DBuf<T> ST, E9, V9, O9, M9, Wq;         // P x P and n x P work
    DBuf<T> FvoT, Ta0;
    DBuf<double> red;                       // reduction scratch
    DBuf<int> flag;
    DBuf<unsigned long long> chk;           // symmetry / finiteness check results

    // Slab scratch.
    DBuf<T> Lh_oo, Lh_vv, Lh_vo, dtr, Wfo, Wfv;
    DBuf<T> M1, Bbar, N1, Btil, C1, D1, M2, M3, E, TA, W, M4, D8, M5, Mo;

    // Alg. 6 scratch (C6, D6, Ech, Fch, H, M6, I6 hold one block of x6 X's).
    DBuf<T> A6, C6, D6, Ech, Fch, Gch, H, M6, I6;
    // Float64-accurate triangle on the FP32 pipe (float64 engine, tensor-core
    // policy): E and F as float pairs with interleaved row pairs; G_I^YZ
    // (Gall or Gch) is replaced in place by its float pairs.
    bool tri_df = false;
    // Mixed triangle over X pairs in packed lanes (C_i, D_a, E, F with the rows
    // of a pair interleaved, slabs of an even number of rows).
    bool tri_pair = false;
    DBuf<float4> E4, F4;
    // Alg. 7 scratch (C7, D7: P x G on the dense route, G x P transposed on
    // the blocked route).
    DBuf<T> R7, S7, C7, D7, Yv, M7, Yo, N7, E7, P7, G7;
    bool alg7_dense = false;
    // Algs. 4 and 5 (O(N^5) route for Eqs. 32-33)
    bool t2sq_n5 = false;
    int nb45 = 0;                           // pairs per batched product
    DBuf<T> Q4, S5;                         // o x v x P: W_i T;  v x o x P: U_a T
    DBuf<T> C45, M245, D45, M345, F45, M445, G45, M545, I45, R45;
    DBuf<T> Kx;                             // (ov) x (ov): Kx[(ia),(jb)] = (ib|ja)
    DBuf<T> W7;                             // P x (ov)

    // init = init_begin, load_cholesky of all K vectors, init_finish; with
    // L == nullptr it stops after init_begin and the caller supplies the
    // vectors (pending until init_finish).
    Err init(const thc_config& cfg, const double* eps_o, const double* eps_v,
             const double* Y, const double* L, const double* xin, const double* zin,
             cudaStream_t s);
    Err init_begin(const thc_config& cfg, const double* eps_o, const double* eps_v,
                   const double* Y, const double* xin, const double* zin, cudaStream_t s);
    // Cholesky vectors k0 .. k0 + nk - 1 (nk x n x n float64, host or device).
    Err load_cholesky(int k0, int nk, const double* L);
    Err init_finish();
    bool pending = false;                   // Cholesky vectors still arriving
    thc_config cfg0{};
    std::vector<char> loaded;               // per Cholesky vector
    DBuf<double> lstage;                    // float64 staging of kb vectors
    DBuf<T> lstageT;
    Err residual(const double* Zc, const double* t1in, double* sigmaZ, double* sigma1,
                 double* energy);
    Err energy(const double* Zc, const double* t1in, double* e);

    // Device-resident variant used by the solver: Tc and t1 already loaded.
    Err residual_dev(bool want_energy);
    Err energy_dev();

    Err load(const double* src, T* dst, long long count);
    // THC_ERR_ARG if |a - a^T| > rel max|a|, THC_ERR_NUMERIC if a is not finite
    // (a: n x n float64 in device memory).
    Err check_sym(const double* a, int n, double rel, const char* what);
    Err check_finite(const double* a, long long count, const char* what);
    Err set_state(const double* Zc, const double* t1in);
    Err mm(int M, int N, int Kd, View<T> A, View<T> B, T* C, long long ldc,
           double alpha, double beta, int batch = 1, long long sAb = 0,
           long long sBb = 0, long long sCb = 0, bool reduce = false);
    Err dress(const T* oo_, const T* ov_, const T* vv_, int nb, T* out_oo, T* out_vv,
              T* out_vo);
    Err fock_slab(int nb, const T* Loo_, const T* Lov_, const T* Lvo_, const T* Lvv_);
    Err d_operator(const T* M, int nb, T* Dout);
    Err alg6(T* sgm);
    Err alg45(T* sgm);
    // MP2-like one-particle density matrices of the amplitudes encoded by the
    // THC core Zc (App. II, Eqs. 49-56); D_oo (o x o), D_vv (v x v) float64.
    Err mp2_density(const double* Zc, double* Doo_out, double* Dvv_out);
    DBuf<T> dn_x1, dn_x2, dn_c, dn_m1, dn_m2, dn_q, dn_ones, dn_oo, dn_vv, dn_t1;
    DBuf<double> dn_out;
    Err alg7(T* sgm);
};

}  // namespace thc
