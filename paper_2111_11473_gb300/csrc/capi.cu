// C ABI of the THC-RR-CCSD library (declared in include/thc.h).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <new>
#include <string>
#include <algorithm>

#include "engine.cuh"
#include "solver.cuh"

struct thc_mlp {
    thc::Mlp m;
    std::string err;
    ~thc_mlp() { m.destroy(); }
};

struct thc_ctx {
    thc_config cfg{};
    cudaStream_t st = nullptr;
    std::string err;
    std::unique_ptr<thc::Engine<double>> e64;
    std::unique_ptr<thc::Engine<float>> e32;
    std::unique_ptr<thc::Solver> solver;
};

namespace {

thread_local std::string g_init_error;

thc_status fail(thc_ctx* c, const thc::Err& e) {
    if (c && c->err.empty()) c->err = e.msg;
    return e.code;
}

thc::Err check_config(const thc_config* cfg) {
    if (!cfg) return {THC_ERR_ARG, "cfg is NULL"};
    if (cfg->n_occ <= 0 || cfg->n_vir <= 0 || cfg->n_p <= 0 || cfg->n_g <= 0 || cfg->n_k <= 0)
        return {THC_ERR_ARG, "every dimension must be positive"};
    if (cfg->precision != THC_PREC_FP64 && cfg->precision != THC_PREC_MIXED &&
        cfg->precision != THC_PREC_FP64_TC)
        return {THC_ERR_ARG, "unknown precision policy"};
    if (cfg->k_slab < 0 || cfg->i_chunk < 0 || cfg->x_block < 0 || cfg->x_block6 < 0)
        return {THC_ERR_ARG, "blocking sizes must be >= 0"};
    if (cfg->tc_products != 0 && cfg->tc_products != 1 && cfg->tc_products != 3)
        return {THC_ERR_ARG, "tc_products must be 0, 1 or 3"};
    if (cfg->alg7_route < 0 || cfg->alg7_route > 2)
        return {THC_ERR_ARG, "alg7_route must be 0, 1 or 2"};
    if (cfg->t2sq_route < 0 || cfg->t2sq_route > 2)
        return {THC_ERR_ARG, "t2sq_route must be 0, 1 or 2"};
    if (cfg->shard_count < 0 || cfg->shard_count > cfg->n_k || cfg->shard_index < 0 ||
        (cfg->shard_count <= 1 ? cfg->shard_index != 0 : cfg->shard_index >= cfg->shard_count))
        return {THC_ERR_ARG, "shard_index must lie in 0 .. shard_count - 1, shard_count <= n_k"};
    const bool f64 = cfg->precision != THC_PREC_MIXED;
    for (int s = 0; s < THC_N_STEPS; ++s) {
        const int p = cfg->policy[s];
        if (p == THC_POL_DEFAULT) continue;
        const bool ok = f64 ? (p == THC_POL_FP64 || p == THC_POL_FP64_TC)
                            : (s == THC_STEP_TRIANGLE ? p == THC_POL_FP32
                                                      : (p == THC_POL_BF16X3 || p == THC_POL_BF16 ||
                                                         p == THC_POL_FP32));
        if (!ok)
            return {THC_ERR_ARG, std::string("policy of step ") + thc_step_name(s) +
                                     " does not fit the context's precision"};
    }
    return {};
}

// The solver of a context, set up on first use.
thc::Err solver_of(thc_ctx* c) {
    if (c->solver) return {};
    c->solver.reset(new thc::Solver());
    thc::Err e = c->e64 ? c->solver->setup(*c->e64, c->cfg.lsq_rel_cutoff)
                        : c->solver->setup(*c->e32, c->cfg.lsq_rel_cutoff);
    if (!e.ok()) c->solver.reset();
    return e;
}

// Calls that evaluate anything need the Cholesky vectors in place.
thc::Err ready(const thc_ctx* c) {
    const bool pend = c->e64 ? c->e64->pending : c->e32->pending;
    if (pend)
        return {THC_ERR_ARG, "the context waits for its Cholesky vectors (thc_load_cholesky, "
                             "thc_init_finish)"};
    return {};
}

}  // namespace

namespace thc {
void set_thread_error(const std::string& msg) { g_init_error = msg; }

namespace {
std::atomic<long long> g_fail_alloc_left{0};
std::atomic<bool> g_poison{false};
std::atomic<bool> g_products{false};
}  // namespace

void debug_arm_from_env() {
    const char* f = std::getenv("THC_FAIL_ALLOC_AT");
    g_fail_alloc_left = f ? std::max(0LL, std::atoll(f)) : 0LL;
    const char* q = std::getenv("THC_POISON_WORKSPACE");
    g_poison = q && q[0] && q[0] != '0';
    const char* d = std::getenv("THC_DEBUG_PRODUCTS");
    g_products = d && d[0] && d[0] != '0';
}

bool debug_alloc_fails() {
    long long left = g_fail_alloc_left.load();
    while (left > 0) {
        if (g_fail_alloc_left.compare_exchange_weak(left, left - 1)) return left == 1;
    }
    return false;
}

bool debug_poison() { return g_poison.load(); }
bool debug_products() { return g_products.load(); }
}  // namespace thc

extern "C" {

thc_status thc_config_default(thc_config* cfg, int n_occ, int n_vir, int n_p, int n_g,
                              int n_k) {
    if (!cfg) return THC_ERR_ARG;
    *cfg = thc_config{};
    cfg->n_occ = n_occ;
    cfg->n_vir = n_vir;
    cfg->n_p = n_p;
    cfg->n_g = n_g;
    cfg->n_k = n_k;
    cfg->precision = THC_PREC_FP64;
    cfg->lsq_rel_cutoff = 1e-10;
    cfg->tc_products = 3;
    return check_config(cfg).code;
}

thc_status thc_solve_opts_default(thc_solve_opts* opts) {
    if (!opts) return THC_ERR_ARG;
    opts->r_tol = 1e-8;
    opts->e_tol = 0.0;
    opts->max_iter = 100;
    opts->diis_n = 8;
    opts->use_mlp = 0;
    opts->verbose = 0;
    opts->history = nullptr;
    opts->mlp = nullptr;
    opts->record_pairs = 0;
    opts->record_seed = 0;
    opts->resume = 0;
    opts->mlp_accept = 0;
    opts->mlp_blocks = 3;
    return THC_OK;
}

thc_status thc_init(const thc_config* cfg, const double* eps_occ, const double* eps_vir,
                    const double* Y, const double* L, const double* x, const double* z,
                    void* stream, thc_ctx** out) {
    g_init_error.clear();
    if (!out) { g_init_error = "out is NULL"; return THC_ERR_ARG; }
    *out = nullptr;
    thc::debug_arm_from_env();
    thc::Err e = check_config(cfg);
    if (e.ok() && (!eps_occ || !eps_vir || !Y || !x || !z))
        e = {THC_ERR_ARG, "an input pointer is NULL"};
    if (!e.ok()) { g_init_error = e.msg; return e.code; }
    thc_ctx* c = new (std::nothrow) thc_ctx;
    if (!c) { g_init_error = "host allocation failed"; return THC_ERR_OOM; }
    c->cfg = *cfg;
    if (c->cfg.lsq_rel_cutoff <= 0) c->cfg.lsq_rel_cutoff = 1e-10;
    c->st = (cudaStream_t)stream;
    {
        if (cfg->precision != THC_PREC_MIXED) {
            c->e64.reset(new thc::Engine<double>());
            e = c->e64->init(c->cfg, eps_occ, eps_vir, Y, L, x, z, c->st);
        } else {
            c->e32.reset(new thc::Engine<float>());
            e = c->e32->init(c->cfg, eps_occ, eps_vir, Y, L, x, z, c->st);
        }
    }
    if (!e.ok()) {
        g_init_error = e.msg;
        delete c;
        return e.code;
    }
    *out = c;
    return THC_OK;
}

thc_status thc_load_cholesky(thc_ctx* c, int k0, int nk, const double* L) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    thc::Err e = c->e64 ? c->e64->load_cholesky(k0, nk, L) : c->e32->load_cholesky(k0, nk, L);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_init_finish(thc_ctx* c) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    thc::Err e = c->e64 ? c->e64->init_finish() : c->e32->init_finish();
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_residual(thc_ctx* c, const double* Zc, const double* t1, double* sigmaZ,
                        double* sigma1, double* energy) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    if (thc::Err r = ready(c); !r.ok()) return fail(c, r);
    if (!Zc || !t1 || !sigmaZ || !sigma1) return fail(c, {THC_ERR_ARG, "NULL argument"});
    thc::Err e = c->e64 ? c->e64->residual(Zc, t1, sigmaZ, sigma1, energy)
               : c->e32->residual(Zc, t1, sigmaZ, sigma1, energy);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_energy(thc_ctx* c, const double* Zc, const double* t1, double* energy) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    if (thc::Err r = ready(c); !r.ok()) return fail(c, r);
    if (!Zc || !t1 || !energy) return fail(c, {THC_ERR_ARG, "NULL argument"});
    thc::Err e = c->e64 ? c->e64->energy(Zc, t1, energy) : c->e32->energy(Zc, t1, energy);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_mp2_density(thc_ctx* c, const double* Zc, double* D_oo, double* D_vv) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    if (thc::Err r = ready(c); !r.ok()) return fail(c, r);
    if (!Zc || !D_oo || !D_vv) return fail(c, {THC_ERR_ARG, "NULL argument"});
    thc::Err e = c->e64 ? c->e64->mp2_density(Zc, D_oo, D_vv)
                        : c->e32->mp2_density(Zc, D_oo, D_vv);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_solve(thc_ctx* c, const thc_solve_opts* opts, double* Zc_inout,
                     double* t1_inout, thc_report* report) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    if (thc::Err r = ready(c); !r.ok()) return fail(c, r);
    if (!opts || !Zc_inout || !t1_inout) return fail(c, {THC_ERR_ARG, "NULL argument"});
    if (c->cfg.shard_count > 1)
        return fail(c, {THC_ERR_UNSUPPORTED, "thc_solve needs the whole residual: a sharded "
                                             "context evaluates one shard"});
    if (opts->mlp_accept < 0 || opts->mlp_accept > 2)
        return fail(c, {THC_ERR_ARG, "mlp_accept must be 0, 1 or 2"});
    if (opts->mlp_blocks < 0 || opts->mlp_blocks > 3)
        return fail(c, {THC_ERR_ARG, "mlp_blocks must be 0 .. 3"});
    if (thc::Err e = solver_of(c); !e.ok()) return fail(c, e);
    thc_report rep{};
    thc::Mlp* mlp = opts->mlp ? &opts->mlp->m : nullptr;
    if (mlp) mlp->st = c->st;
    thc::Err e = c->e64 ? c->solver->run(*c->e64, *opts, Zc_inout, t1_inout, &rep, mlp)
                        : c->solver->run(*c->e32, *opts, Zc_inout, t1_inout, &rep, mlp);
    if (report) *report = rep;
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_solve_state_size(thc_ctx* c, size_t* bytes) {
    if (!c || !bytes) return THC_ERR_ARG;
    c->err.clear();
    if (!c->solver || !c->solver->resumable)
        return fail(c, {THC_ERR_ARG, "no stopped plain solve in this context"});
    *bytes = c->solver->state_bytes();
    return THC_OK;
}

thc_status thc_solve_state_save(thc_ctx* c, void* buf, size_t bytes) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    if (!c->solver) return fail(c, {THC_ERR_ARG, "no stopped plain solve in this context"});
    thc::Err e = c->solver->state_save(buf, bytes, c->st);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_solve_state_load(thc_ctx* c, const void* buf, size_t bytes) {
    if (!c) return THC_ERR_ARG;
    c->err.clear();
    if (thc::Err r = ready(c); !r.ok()) return fail(c, r);
    if (thc::Err e = solver_of(c); !e.ok()) return fail(c, e);
    thc::Err e = c->solver->state_load(buf, bytes, c->st);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

thc_status thc_profile_enable(thc_ctx* c, int on) {
    if (!c) return THC_ERR_ARG;
    thc::Profiler& p = c->e64 ? c->e64->prof : c->e32->prof;
    p.on = on != 0;
    p.reset();
    p.marks.clear();
    p.used = 0;
    p.cur = -1;
    return THC_OK;
}

thc_status thc_profile_read(thc_ctx* c, thc_profile* out) {
    if (!c || !out) return THC_ERR_ARG;
    const thc::Profiler& p = c->e64 ? c->e64->prof : c->e32->prof;
    for (int i = 0; i < THC_N_STEPS; ++i) {
        out->ms[i] = p.ms[i];
        out->flops[i] = p.flops[i];
        out->launches[i] = p.launches[i];
    }
    out->residuals = p.residuals;
    out->kernel_launches = p.kernel_launches;
    return THC_OK;
}

const char* thc_step_name(int step) {
    static const char* names[THC_N_STEPS] = {"dress", "fock", "alg1", "alg2_8", "post",
                                             "alg6_gemm", "triangle", "alg6_post", "alg7",
                                             "energy"};
    if (step < 0 || step >= THC_N_STEPS) return nullptr;
    return names[step];
}

thc_status thc_solve_pairs(thc_ctx* c, float* X, float* j, float* t, long long max_n,
                           long long* n_out) {
    if (!c || !n_out) return THC_ERR_ARG;
    if (!c->solver) { *n_out = 0; return THC_OK; }
    thc::Err e = c->solver->pairs(X, j, t, max_n, n_out, c->st);
    if (!e.ok()) return fail(c, e);
    return THC_OK;
}

// Device copies of possibly-host arrays for the network entry points.
struct DevArr {
    float* p = nullptr;
    bool own = false;
    ~DevArr() { if (own && p) cudaFree(p); }
};

// Kernels only ever see device allocations: a caller's pointer is used in
// place only if the runtime reports it as device memory; host memory of any
// kind (pageable, pinned, managed or system-allocated) is staged through a
// device copy.
static thc::Err dev_in(const float* src, long long n, cudaStream_t st, DevArr& out) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess && a.type == cudaMemoryTypeDevice &&
        a.devicePointer == (const void*)src) {
        out.p = const_cast<float*>(src);
        return {};
    }
    cudaGetLastError();
    THC_CUDA(cudaMalloc(&out.p, sizeof(float) * std::max<long long>(n, 1)));
    out.own = true;
    THC_CUDA(cudaMemcpyAsync(out.p, src, sizeof(float) * n, cudaMemcpyDefault, st));
    return {};
}

thc_status thc_mlp_create(int hidden, unsigned long long seed, int bf16, void* stream,
                          thc_mlp** out) {
    if (!out || hidden <= 0 || hidden % 16) {
        g_init_error = "thc_mlp_create: hidden must be a positive multiple of 16";
        return THC_ERR_ARG;
    }
    *out = nullptr;
    thc_mlp* m = new (std::nothrow) thc_mlp;
    if (!m) return THC_ERR_OOM;
    thc::Err e = m->m.create(hidden, seed, bf16 != 0, (cudaStream_t)stream);
    if (!e.ok()) { g_init_error = e.msg; delete m; return e.code; }
    *out = m;
    return THC_OK;
}

thc_status thc_mlp_num_params(const thc_mlp* m, long long* n) {
    if (!m || !n) return THC_ERR_ARG;
    *n = m->m.np;
    return THC_OK;
}

thc_status thc_mlp_get_params(thc_mlp* m, float* params) {
    if (!m || !params) return THC_ERR_ARG;
    if (cudaMemcpy(params, m->m.theta, sizeof(float) * m->m.np, cudaMemcpyDefault) != cudaSuccess)
        return THC_ERR_CUDA;
    return THC_OK;
}

thc_status thc_mlp_set_params(thc_mlp* m, const float* params) {
    if (!m || !params) return THC_ERR_ARG;
    if (cudaMemcpy(m->m.theta, params, sizeof(float) * m->m.np, cudaMemcpyDefault) != cudaSuccess)
        return THC_ERR_CUDA;
    cudaMemset(m->m.m, 0, sizeof(float) * m->m.np);
    cudaMemset(m->m.v, 0, sizeof(float) * m->m.np);
    m->m.step = 0;
    return THC_OK;
}

thc_status thc_mlp_predict(thc_mlp* m, const float* X, long long n, float* y) {
    if (!m || !X || !y || n <= 0) return THC_ERR_ARG;
    DevArr dx, dy;
    thc::Err e = dev_in(X, n * thc::kMlpFeatures, m->m.st, dx);
    if (e.ok()) e = dev_in(y, n, m->m.st, dy);
    if (e.ok()) e = m->m.forward(dx.p, n, dy.p);
    if (e.ok() && dy.own)
        if (cudaMemcpyAsync(y, dy.p, sizeof(float) * n, cudaMemcpyDefault, m->m.st) != cudaSuccess)
            e = {THC_ERR_CUDA, "copy-out failed"};
    if (e.ok() && cudaStreamSynchronize(m->m.st) != cudaSuccess) e = {THC_ERR_CUDA, "sync failed"};
    if (!e.ok()) { g_init_error = e.msg; return e.code; }
    return THC_OK;
}

thc_status thc_mlp_loss_grad(thc_mlp* m, const float* X, const float* j, const float* t,
                             long long n, double* loss, float* grad) {
    if (!m || !X || !j || !t || n <= 0) return THC_ERR_ARG;
    DevArr dx, dj, dt;
    thc::Err e = dev_in(X, n * thc::kMlpFeatures, m->m.st, dx);
    if (e.ok()) e = dev_in(j, n, m->m.st, dj);
    if (e.ok()) e = dev_in(t, n, m->m.st, dt);
    double l = 0;
    if (e.ok()) e = m->m.loss_grad(dx.p, dj.p, dt.p, n, &l);
    if (e.ok() && grad &&
        cudaMemcpy(grad, m->m.grad, sizeof(float) * m->m.np, cudaMemcpyDefault) != cudaSuccess)
        e = {THC_ERR_CUDA, "copy-out failed"};
    if (!e.ok()) { g_init_error = e.msg; return e.code; }
    if (loss) *loss = l;
    return THC_OK;
}

thc_status thc_mlp_train(thc_mlp* m, const float* X, const float* j, const float* t,
                         long long n, int epochs, int batch, double lr,
                         unsigned long long seed, double* final_loss) {
    if (!m || !X || !j || !t || n <= 0) return THC_ERR_ARG;
    DevArr dx, dj, dt;
    thc::Err e = dev_in(X, n * thc::kMlpFeatures, m->m.st, dx);
    if (e.ok()) e = dev_in(j, n, m->m.st, dj);
    if (e.ok()) e = dev_in(t, n, m->m.st, dt);
    if (e.ok()) e = m->m.train(dx.p, dj.p, dt.p, n, epochs, batch, (float)lr, seed, final_loss);
    if (e.ok() && cudaStreamSynchronize(m->m.st) != cudaSuccess) e = {THC_ERR_CUDA, "sync failed"};
    if (!e.ok()) { g_init_error = e.msg; return e.code; }
    return THC_OK;
}

void thc_mlp_destroy(thc_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->m.st);
    delete m;
}

thc_status thc_selftest_gemm(int cases, unsigned long long seed, double* max_rel_err,
                             int* failures, void* stream) {
    if (cases < 0) return THC_ERR_ARG;
    double mr = 0;
    int nf = 0;
    cudaError_t e = thc::gemm_tc_selftest(cases, seed, &mr, &nf, (cudaStream_t)stream);
    if (max_rel_err) *max_rel_err = mr;
    if (failures) *failures = nf;
    if (e != cudaSuccess) {
        g_init_error = std::string("thc_selftest_gemm: ") + cudaGetErrorString(e);
        return THC_ERR_CUDA;
    }
    if (nf) {
        g_init_error = "thc_selftest_gemm: " + std::to_string(nf) + " case(s) outside the bound";
        return THC_ERR_NUMERIC;
    }
    return THC_OK;
}

thc_status thc_selftest_gemm_f64(int cases, unsigned long long seed, double* max_rel,
                                 int* failures, void* stream) {
    if (cases < 0) return THC_ERR_ARG;
    double mr = 0;
    int nf = 0;
    cudaError_t e = thc::gemm_f64_tc_selftest(cases, seed, &mr, &nf, (cudaStream_t)stream);
    if (max_rel) *max_rel = mr;
    if (failures) *failures = nf;
    if (e != cudaSuccess) {
        g_init_error = std::string("thc_selftest_gemm_f64: ") + cudaGetErrorString(e);
        return THC_ERR_CUDA;
    }
    if (nf) {
        g_init_error = "thc_selftest_gemm_f64: " + std::to_string(nf) + " case(s) outside the bound";
        return THC_ERR_NUMERIC;
    }
    return THC_OK;
}

thc_status thc_selftest_bounded_wait(int complete, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int* flag = nullptr;
    int h = 0;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    // about 1 ms at 2 GHz
    if (e == cudaSuccess) e = thc::wait_selftest(complete, 2000000LL, flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (flag) cudaFree(flag);
    if (e != cudaSuccess) {
        g_init_error = std::string("thc_selftest_bounded_wait: ") + cudaGetErrorString(e);
        return THC_ERR_CUDA;
    }
    if (h) {
        g_init_error = "thc_selftest_bounded_wait: the bounded wait expired";
        return THC_ERR_TIMEOUT;
    }
    return THC_OK;
}

const char* thc_last_error(const thc_ctx* c) {
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

void thc_destroy(thc_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    delete c;
}

}  // extern "C"
