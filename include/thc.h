/*
 * thc.h - C ABI of the GB300 THC-RR-CCSD residual library (libthc.so).
 *
 * The library evaluates the residual of rank-reduced coupled-cluster singles
 * and doubles with tensor-hypercontracted doubles amplitudes (Hohenstein,
 * Fales, Parrish, Martinez, "Rank-reduced coupled-cluster III", Sec. II-III):
 *
 *   t_ij^ab = sum_WX y_i^W y_a^W Zc^WX y_j^X y_b^X                    (Eq. 23)
 *   (pq^|rs) = sum_A L^_pq^A L^_rs^A, L^ = T1-dressed Cholesky vectors (Eqs. 24-27)
 *   (ia|jb)  = sum_IJ x_i^I x_a^I z^IJ x_j^J x_b^J                    (Eq. 17)
 *
 * and returns the doubles residual projected onto the amplitude factors,
 *   sigma^WX = sum_ijab y_i^W y_a^W y_j^X y_b^X Omega_ij^ab       (Eq. 6, Eq. 14)
 * (the sum of Eqs. 28, 29, 31, 34, 35 and 41), the singles residual
 * Omega_i^a (Eqs. 38 and 42), and the closed-shell CCSD energy.
 *
 * Conventions shared by every entry point
 *   - All arrays are row-major IEEE float64 (C order), whatever the internal
 *     precision policy.
 *   - Orbitals: o occupied then v virtual, n = o + v.  Y is n x P with the
 *     occupied rows first; x is n x G likewise; L is K x n x n.
 *   - Pointers may be host or device memory (the kind is detected per
 *     pointer); outputs are written into the caller's buffer in its own
 *     memory kind.  Every call is synchronous on the context's stream: when it
 *     returns, outputs are complete and inputs may be reused.
 *   - Every call returns a thc_status; nothing throws across the ABI.  On
 *     failure thc_last_error() describes the first error on that context.
 *   - A context belongs to one GPU and one stream and is not thread-safe;
 *     separate contexts are independent.
 *
 * Debugging environment variables, read at every thc_init:
 *   THC_FAIL_ALLOC_AT=n     the n-th device allocation from then on fails
 *                           with THC_ERR_OOM (failure injection);
 *   THC_POISON_WORKSPACE=1  every scratch buffer is filled with NaN bytes at
 *                           the end of initialisation, so a read of scratch
 *                           that has not been written shows up as a
 *                           non-finite result;
 *   THC_DEBUG_PRODUCTS=1    every product of at least 3e7 flops that runs on
 *                           the CUDA cores although a tensor-core path is
 *                           enabled is reported on stderr with the reason.
 */
#ifndef THC_H
#define THC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thc_ctx thc_ctx;

typedef enum {
    THC_OK = 0,
    THC_ERR_ARG = 1,            /* bad dimension, null pointer, asymmetric input */
    THC_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    THC_ERR_OOM = 3,            /* device workspace could not be allocated */
    THC_ERR_NUMERIC = 4,        /* non-finite input/output, metric not positive */
    THC_ERR_NOT_CONVERGED = 5,  /* thc_solve hit max_iter */
    THC_ERR_TIMEOUT = 6,        /* a bounded device wait expired */
    THC_ERR_UNSUPPORTED = 7     /* feature not available on this device */
} thc_status;

/* Arithmetic policy for the bulk contractions.  FP64: every step in float64
 * on the CUDA cores.  MIXED: operands stored in float32, tensor-core GEMMs
 * with split (hi/lo) bf16 products and float32 accumulation, float32
 * CUDA-core triangle kernel; the sigma accumulation, energy, least squares
 * and DIIS stay float64.  FP64_TC: float64 storage and arithmetic as FP64,
 * but the products of at least 3e7 flops (those a cost model of the two
 * paths does not keep on the CUDA cores) run on the tensor cores as exact
 * integer products of 8 slices of 7 bits per operand row (scaled by a power
 * of two per row), combined in float64: each product term is within about
 * 1.2e-16 of its row and column scale, float64 rounding level; the triangle
 * (Alg. 6 line 11) runs in float pairs on the FP32 pipe, each term within
 * about 2^-45 of |E F G|.  Per-step choices: thc_config.policy. */
typedef enum { THC_PREC_FP64 = 0, THC_PREC_MIXED = 1, THC_PREC_FP64_TC = 2 } thc_precision;

/* Steps of one residual evaluation (per-step policy, timing and flop counts). */
enum {
    THC_STEP_DRESS = 0,      /* T1 dressing of the Cholesky vectors (Eqs. 25-27) */
    THC_STEP_FOCK = 1,       /* Coulomb/exchange parts of the dressed Fock matrix */
    THC_STEP_ALG1 = 2,       /* ladders, Alg. 1 (+ Alg. 3 intermediate) */
    THC_STEP_ALG2_8 = 3,     /* Alg. 2 and Alg. 8 per Cholesky vector */
    THC_STEP_POST = 4,       /* Alg. 2/3 closing products, Algs. 9 and 10 */
    THC_STEP_ALG6_GEMM = 5,  /* Alg. 6 lines 1-10 (contractions) */
    THC_STEP_TRIANGLE = 6,   /* Alg. 6 line 11 (triangle kernel) */
    THC_STEP_ALG6_POST = 7,  /* Alg. 6 lines 13-16 */
    THC_STEP_ALG7 = 8,       /* Alg. 7 */
    THC_STEP_ENERGY = 9,     /* energy */
    THC_N_STEPS = 10
};

/* Arithmetic of one step (thc_config.policy[step]); 0 = the context's
 * precision policy.  Float64 contexts (THC_PREC_FP64, THC_PREC_FP64_TC):
 *   THC_POL_FP64     float64 products and triangle on the CUDA cores
 *   THC_POL_FP64_TC  products of at least 3e7 flops as exact integer slices
 *                    on the tensor cores (float64 accuracy); the triangle
 *                    (Alg. 6 line 11, THC_STEP_TRIANGLE) in float pairs with
 *                    error-free transformations on the FP32 pipe, about
 *                    2^-45 of |E F G| per term
 * Mixed contexts (THC_PREC_MIXED, float32 storage):
 *   THC_POL_BF16X3   products as bf16 hi*hi + hi*lo + lo*hi on the tensor
 *                    cores, float32 accumulation
 *   THC_POL_BF16     bf16 hi*hi only (about 2^-8 per factor)
 *   THC_POL_FP32     float32 products on the CUDA cores
 * The triangle of a mixed context is the float32 kernel (DEFAULT or FP32
 * only).  A value outside the context's family is THC_ERR_ARG.  Products
 * outside the residual's steps (initialisation, thc_mp2_density) follow the
 * context's policy. */
enum {
    THC_POL_DEFAULT = 0,
    THC_POL_FP64 = 1,
    THC_POL_FP64_TC = 2,
    THC_POL_BF16X3 = 3,
    THC_POL_BF16 = 4,
    THC_POL_FP32 = 5
};

typedef struct {
    int n_occ;               /* o > 0 */
    int n_vir;               /* v > 0 */
    int n_p;                 /* P: amplitude THC rank (columns of Y) */
    int n_g;                 /* G: ERI-THC grid size (columns of x) */
    int n_k;                 /* K: number of Cholesky vectors */
    int precision;           /* thc_precision */
    int k_slab;              /* Cholesky vectors per fused slab, 0 = auto */
    int i_chunk;             /* grid points per Alg. 6 chunk, 0 = auto */
    int x_block;             /* amplitude-THC columns per Alg. 7 block, 0 = auto */
    size_t workspace_bytes;  /* device workspace limit, 0 = auto */
    double lsq_rel_cutoff;   /* drop metric eigenvalues below cutoff*max (1e-10) */
    int tc_products;         /* MIXED only: tensor-core products per contraction,
                                3 = bf16 hi*hi + hi*lo + lo*hi (default),
                                1 = bf16 hi*hi, 0 = float32 CUDA cores */
    int alg7_route;          /* exchange part of Alg. 7 (Eq. 37): 0 = automatic,
                                1 = through the THC factors as printed (G x G
                                intermediates per X), 2 = through the dense
                                (ib|ja) matrix, (ov)^2 words, built once at init
                                from the THC factors; automatic picks 2 when
                                that matrix takes at most 16 GiB */
    int t2sq_route;          /* T2^2 contributions to Omega^A and Omega^C
                                (Eqs. 32-33): 0 = automatic, 1 = Alg. 6
                                (O(N^4), triangle kernel on the CUDA cores),
                                2 = Algs. 4 and 5 (O(N^5), batched products
                                only); automatic compares the estimated time
                                of both at the context's precision */
    int x_block6;            /* amplitude-THC indices X per Alg. 6 block: H,
                                C_i, D_a, E and F are formed for one block of
                                X rows at a time (G_I^YZ is shared); 0 = auto:
                                all P rows when H (P^3 words), D_a and C_i fit
                                a quarter of the free memory (at most 48 GiB),
                                else the fewest blocks that do, rounded up to
                                32 rows */
    int policy[THC_N_STEPS]; /* per-step arithmetic, THC_POL_* (0 = default) */
    int shard_index;         /* this context's shard, 0 .. shard_count - 1 */
    int shard_count;         /* > 1: the context evaluates one shard of the
                                residual (Sec. III's multi-GPU split): the
                                Cholesky vectors [K s/n, K (s+1)/n) for Algs.
                                1, 2, 3, 8, the Fock matrix and the singles
                                energy, the amplitude indices X in
                                [P s/n, P (s+1)/n) for Alg. 6, Alg. 7 on the
                                last shard, the orbital-energy Fock terms on
                                the first.  thc_residual and thc_energy then
                                return that shard's part: the sums of sigmaZ,
                                sigma1 and the energy over all shards are the
                                unsharded results (every step is linear in
                                these partial sums).  Only the shard's own
                                Cholesky vectors are stored.  thc_solve is not
                                available on a sharded context.  0 or 1 =
                                unsharded; needs shard_count <= n_k. */
} thc_config;

/* Fill *cfg with defaults for the given sizes (FP64, automatic blocking). */
thc_status thc_config_default(thc_config* cfg, int n_occ, int n_vir, int n_p,
                              int n_g, int n_k);

/*
 * thc_init - copy the system to the device and precompute the fixed parts.
 *
 *   eps_occ  o      occupied orbital energies (canonical Hartree-Fock: the
 *                   Fock matrix is diag(eps); the core Hamiltonian is
 *                   recovered from it and the Cholesky integrals)
 *   eps_vir  v      virtual orbital energies
 *   Y        n x P  amplitude collocation factors y_p^W (Eq. 7, Eq. 23)
 *   L        K x n x n  Cholesky vectors L_pq^A, symmetric in pq (Eq. 24);
 *                   NULL = supplied later by thc_load_cholesky (systems whose
 *                   float64 vectors do not fit one array), after which
 *                   thc_init_finish completes the initialisation
 *   x        n x G  ERI-THC collocation x_p^I (Eq. 17)
 *   z        G x G  ERI-THC core z^IJ, symmetric (Eq. 17)
 *   stream   cudaStream_t to run on, or NULL for the legacy default stream
 *
 * Precomputes o^XY, v^XY (Alg. 1 lines 1-2), the metric S = o*v (Eq. 10)
 * and the orthonormal working basis of Eq. 22 (generalised eigenbasis of
 * the orbital-energy Fock block in the metric).  Inputs are copied; the
 * caller keeps ownership.  Only the lower triangle (q <= p) of each
 * vector's virtual-virtual block is read; it is stored packed.  Errors:
 * THC_ERR_ARG for non-positive sizes or asymmetric z, THC_ERR_OOM,
 * THC_ERR_CUDA, THC_ERR_NUMERIC if the metric has no positive eigenvalue.
 * On failure *out is NULL.
 */
thc_status thc_init(const thc_config* cfg, const double* eps_occ,
                    const double* eps_vir, const double* Y, const double* L,
                    const double* x, const double* z, void* stream,
                    thc_ctx** out);

/*
 * thc_load_cholesky - Cholesky vectors k0 .. k0 + nk - 1 of a context made
 * by thc_init with L = NULL.
 *
 *   L   nk x n x n float64, row-major, symmetric in the last two indices
 *       (host or device; copied before the call returns)
 *
 * Vectors may arrive in any order and any number of calls; a vector loaded
 * twice keeps the second copy.  Errors: THC_ERR_ARG if the range leaves
 * 0 .. K - 1, L is NULL or the context is not waiting for vectors.
 */
thc_status thc_load_cholesky(thc_ctx* ctx, int k0, int nk, const double* L);

/*
 * thc_init_finish - the parts of thc_init that need the Cholesky vectors
 * (energy weight of the core, Alg. 6 and 7 fixed parts, workspaces).  Every
 * other call on the context returns THC_ERR_ARG until it has succeeded.
 * Errors: THC_ERR_ARG if a vector is missing or nothing is pending, and as
 * thc_init.
 */
thc_status thc_init_finish(thc_ctx* ctx);

/*
 * thc_residual - one evaluation of the projected residual (Algs. 1-10).
 *
 *   Zc      P x P  symmetric THC core T^WX (Eq. 22-23), input
 *   t1      o x v  singles t_i^a, input
 *   sigmaZ  P x P  sigma^WX, output (y basis, as produced by Algs. 1-9)
 *   sigma1  o x v  Omega_i^a, output (Algs. 8 and 10)
 *   energy  scalar closed-shell CCSD energy at (Zc, t1); may be NULL
 *
 * Errors: THC_ERR_ARG for NULL required pointers, THC_ERR_NUMERIC if an
 * output is not finite.
 */
thc_status thc_residual(thc_ctx* ctx, const double* Zc, const double* t1,
                        double* sigmaZ, double* sigma1, double* energy);

/*
 * thc_energy - closed-shell CCSD energy
 *   E = sum_iajb [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b)
 * with Cholesky integrals (Sec. II.a: the energy is the usual CCSD one),
 * evaluated in O(K P^2) from the THC core.
 */
thc_status thc_energy(thc_ctx* ctx, const double* Zc, const double* t1,
                      double* energy);

/*
 * thc_mp2_density - one-particle density matrices of the doubles amplitudes
 * encoded by the THC core Zc (App. II, Eqs. 47-48):
 *   D_ij = -2 sum_kab t_ik^ab (2 t_jk^ab - t_jk^ba),
 *   D_ab =  2 sum_ijc t_ij^ac (2 t_ij^bc - t_ji^bc),
 * with t_ij^ab = sum_WX y_i^W y_a^W Zc^WX y_j^X y_b^X, evaluated in O(N^4)
 * through the factorisation of Eqs. 49-56 (the MP2 natural-orbital density
 * when Zc holds MP2 amplitudes).  Zc: P x P symmetric, row-major; D_oo:
 * o x o and D_vv: v x v row-major outputs (host or device).  Replaces the
 * context's stored t1 by zero.  Errors as thc_residual.
 */
thc_status thc_mp2_density(thc_ctx* ctx, const double* Zc, double* D_oo, double* D_vv);

/*
 * Checkpoint of a stopped solve (a plain Jacobi + DIIS thc_solve that ended
 * at max_iter): thc_solve_state_size gives the bytes of the host blob,
 * thc_solve_state_save writes it (next point, DIIS vectors and overlap
 * matrix, iteration count), thc_solve_state_load puts it into a context of
 * the same system (same sizes and working basis), after which thc_solve
 * with resume = 1 continues it.  Errors: THC_ERR_ARG if there is no stopped
 * solve, the buffer is too small, or the blob belongs to another system.
 */
thc_status thc_solve_state_size(thc_ctx* ctx, size_t* bytes);
thc_status thc_solve_state_save(thc_ctx* ctx, void* buf, size_t bytes);
thc_status thc_solve_state_load(thc_ctx* ctx, const void* buf, size_t bytes);

/* Learned preconditioner network (see thc_mlp_create). */
typedef struct thc_mlp thc_mlp;

typedef struct {
    double r_tol;        /* stop when |residual| < r_tol (1e-8) */
    double e_tol;        /* and |dE| < e_tol (0 = not used) */
    int max_iter;        /* iteration cap (100) */
    int diis_n;          /* DIIS subspace size (8), 0 = plain Jacobi */
    int use_mlp;         /* 1 = learned preconditioner proposals */
    int verbose;         /* 1 = one line per iteration on stderr */
    double* history;     /* nullable host array of max_iter x 3 doubles: per
                            iteration (energy, residual norm, seconds since
                            the call started) */
    thc_mlp* mlp;        /* network proposing steps when use_mlp = 1 */
    int record_pairs;    /* > 0: record this many training pairs per
                            iteration (elements drawn with replacement) */
    unsigned long long record_seed;   /* seed of that draw */
    int resume;          /* 1 = continue the last plain Jacobi + DIIS solve of
                            this context where it stopped at max_iter (or the
                            state given to thc_solve_state_load): its next
                            point, DIIS history and iteration count; Zc_inout
                            and t1_inout are then outputs only.  The result is
                            bit-identical to one uninterrupted solve.
                            THC_ERR_ARG with use_mlp or record_pairs, another
                            diis_n, or no stopped solve. */
    int mlp_accept;      /* acceptance rule of the network's proposals:
                            0 = the residual norm must drop by at least the
                            factor the last plain Jacobi + DIIS iteration
                            achieved (default); 1 = any drop; 2 = always
                            accept (for tests of the accepted branch and for
                            diagnostics) */
    int mlp_blocks;      /* blocks whose step the network scales: 1 = singles,
                            2 = doubles, 3 or 0 = both (default); the other
                            block keeps the Jacobi step */
} thc_solve_opts;

typedef struct {
    int iters;
    int mlp_accepted;
    int mlp_rejected;
    double energy;
    double r_norm;
    double wall_s;
} thc_report;

/* Fill *opts with the defaults listed above. */
thc_status thc_solve_opts_default(thc_solve_opts* opts);

/*
 * thc_solve - solve the projected amplitude equations from (Zc, t1).
 *
 * Works in the orthonormal basis of Eq. 22 (T^PQ, Zc = C T C^T): Jacobi
 * step -sigma_q/(e_P+e_Q) on the doubles and -Omega_i^a/(eps_a-eps_i) on
 * the singles, Pulay DIIS, float64 throughout the update.  The residual norm
 * is sqrt(|Omega1|^2 + |C^T sigma C|^2).  Zc_inout and t1_inout hold the
 * start point on entry and the solution on return.  Returns
 * THC_ERR_NOT_CONVERGED (with the last iterate written back) at max_iter.
 */
thc_status thc_solve(thc_ctx* ctx, const thc_solve_opts* opts,
                     double* Zc_inout, double* t1_inout, thc_report* report);

/*
 * Learned preconditioner (an addition to the method: the paper does not
 * specify the amplitude update).  A pointwise MLP over the elements of the
 * solver state [t1 | T] (singles t_i^a and the doubles core T^PQ in the
 * working basis): 8 features -> tanh(W1 x + b1) -> tanh(W2 a1 + b2) ->
 * y = w3 . a2 + b3, width `hidden` (256).  An element's Jacobi step is
 * j = -res/(eP + eQ) with (eP, eQ) = (e_P, e_Q) for doubles (res = sigma_q^PQ)
 * and (-eps_i, eps_a) for singles (res = Omega_i^a); with s the RMS of its
 * block's Jacobi step, its features at iteration k are
 *   eP/2, eQ/2, clip(j/s, 10), clip(dx_prev/s, 10), sign(x) log1p(|x|/s)/5,
 *   log10|r|/10, |eP - eQ|/2, +1 (doubles) or -1 (singles).
 * The proposed step is j (1 + clamp(y, -0.95, 4)) for every element, and
 * DIIS stores the step taken as its error vector.  In thc_solve a proposal is
 * accepted by the rule of thc_solve_opts.mlp_accept (default: only if the
 * next residual norm is smaller than the current one by at least the factor
 * the last plain Jacobi + DIIS iteration achieved); otherwise the plain
 * iterate from the same point is evaluated instead (one extra residual), and
 * after two rejections the solve continues without proposals.
 *
 * Training pairs come from thc_solve with record_pairs > 0: per iteration
 * k >= 2, record_pairs doubles elements and a quarter as many singles
 * elements (drawn with replacement): features X (n x 8), the scaled Jacobi
 * step j/s and the scaled ideal step t = (x* - x_k)/s, x* the converged state.
 * Loss:  L = mean_n (j_n (1 + y_n) - t_n)^2,  trained with Adam.
 * Parameters are one float32 vector [W1 (H x 8) | b1 | W2 (H x H) | b2 | w3 | b3]
 * (row-major).  bf16 = 1 runs the H x H layer on the tensor cores with bf16
 * weights/activations and float32 accumulation.  All pointers may be host or
 * device memory; calls are synchronous on the network's stream.
 */
thc_status thc_mlp_create(int hidden, unsigned long long seed, int bf16, void* stream,
                          thc_mlp** out);
thc_status thc_mlp_num_params(const thc_mlp* mlp, long long* n);
thc_status thc_mlp_get_params(thc_mlp* mlp, float* params);
thc_status thc_mlp_set_params(thc_mlp* mlp, const float* params);
/* y[n] = network(X[n]) for n samples of 8 features. */
thc_status thc_mlp_predict(thc_mlp* mlp, const float* X, long long n, float* y);
/* Loss of the samples and, if grad is not NULL, its gradient (n_params floats). */
thc_status thc_mlp_loss_grad(thc_mlp* mlp, const float* X, const float* j, const float* t,
                             long long n, double* loss, float* grad);
/* Adam (beta 0.9/0.999, eps 1e-8) over `epochs` passes in minibatches of
 * `batch`; *final_loss = mean loss of the last pass. */
thc_status thc_mlp_train(thc_mlp* mlp, const float* X, const float* j, const float* t,
                         long long n, int epochs, int batch, double lr,
                         unsigned long long seed, double* final_loss);
void thc_mlp_destroy(thc_mlp* mlp);

/* Copy the training pairs recorded by the last thc_solve (record_pairs > 0,
 * converged) into X (n x 8), j (n), t (n), at most max_n; *n_out = recorded
 * count.  Any output pointer may be NULL. */
thc_status thc_solve_pairs(thc_ctx* ctx, float* X, float* j, float* t, long long max_n,
                           long long* n_out);

/*
 * Per-step device timing (CUDA events recorded on the context's stream
 * around every step of thc_residual while profiling is on; steps as in
 * THC_STEP_*).  flops counts the algorithmic floating-point operations of
 * the step (2 per multiply-add of every contraction, 5 per (I,X,Y,Z) term of
 * the triangle whatever kernel runs it), so flops / ms is the achieved rate
 * of that step.
 */

typedef struct {
    double ms[THC_N_STEPS];         /* accumulated device time per step */
    double flops[THC_N_STEPS];      /* accumulated algorithmic flops per step */
    long long launches[THC_N_STEPS];/* timed segments (kernel launches for the triangle) */
    long long residuals;            /* residual evaluations profiled */
    long long kernel_launches;      /* library kernels launched while profiling */
} thc_profile;

/* Switch profiling on (1) or off (0); switching on clears the counters. */
thc_status thc_profile_enable(thc_ctx* ctx, int on);
/* Copy the accumulated counters into *out. */
thc_status thc_profile_read(thc_ctx* ctx, thc_profile* out);
/* Name of a step ("dress", "fock", ...), or NULL if out of range. */
const char* thc_step_name(int step);

/*
 * thc_energy_noalloc - the CCSD energy of thc_energy, for callers that may
 * not allocate device memory.  No counterpart in the paper.
 *
 * Some callers cannot call cudaMalloc: a process whose device memory is
 * already reserved by another runtime's pool (a framework's caching
 * allocator holding nearly all of HBM), or a latency-critical loop that
 * must not take an allocation's cost or its risk of failing.  This entry
 * point allocates nothing and needs no context: the caller passes device
 * inputs and an output, and the scratch is a fixed, file-scope device array
 * of THC_NOALLOC_SCRATCH doubles (16 MiB) that every GPU which loads the
 * library holds until the process exits.
 *
 *   Y       n x P  device, amplitude collocation factors (occupied rows first)
 *   Lov     K x o x v  device, occupied-virtual blocks of the Cholesky vectors
 *   Zc      P x P  device, THC core;  t1  o x v  device, singles
 *   energy  host or device scalar, output
 *   stream  cudaStream_t or NULL
 *
 * Needs o*P + P*P + P + o*o + 32*K + 1 <= THC_NOALLOC_SCRATCH; larger sizes,
 * inputs that are not device memory, and inputs on a device other than the
 * current one return THC_ERR_ARG with the reason in thc_last_error(NULL).
 * `stream` must belong to the current device.
 *
 * First call per device.  CUDA loads a library's device code lazily (the
 * default since CUDA 12.2), so the scratch array is committed on a device
 * when the first call there loads this code, not when the library is
 * loaded.  A caller whose memory pool will hold nearly all of HBM should
 * therefore make one call (any valid size) before the pool reserves its
 * memory, or run with CUDA_MODULE_LOADING=EAGER.  The first call also looks
 * up the array's device address (with that device current), so make it
 * before any stream capture.  Later calls allocate nothing.
 *
 * Every call on a device shares the one array and leaves its contents
 * behind: calls whose work overlaps on the GPU (other streams, other
 * threads) race, so serialise them.  Synchronous on `stream`.  Agrees with
 * thc_energy to rounding.  Cost: five small launches per Cholesky vector,
 * run one vector after another; meant for modest sizes.
 */
#define THC_NOALLOC_SCRATCH (1 << 21)
thc_status thc_energy_noalloc(int n_occ, int n_vir, int n_p, int n_k,
                              const double* Y, const double* Lov,
                              const double* Zc, const double* t1,
                              double* energy, void* stream);

/*
 * thc_cp_als - eigenvalue-weighted CP factorisation of the rank-reduced
 * projectors (Eqs. 15-16, App. I): U_ia^P ~ sum_W y_i^W y_a^W tau^PW,
 * minimising f = sum_P eps_P^2 sum_ia (U_ia^P - sum_W y_i^W y_a^W tau^PW)^2
 * by `iters` sweeps of alternating least squares (y_o, then y_v, then tau;
 * the y_o update is Eq. 16), float64 on the device.  The W x W normal
 * equations are solved by Cholesky factorisation (App. I uses CG).
 *   U: (n_occ n_vir) x n_rr row-major, row (i, a) = i n_vir + a
 *   eps: n_rr projector eigenvalues (any sign)
 *   y_o: n_occ x rank, y_v: n_vir x rank, tau: n_rr x rank, row-major; the
 *        start point on entry, the result on return
 *   objective: nullable host array of `iters` doubles, f after every sweep
 * All arrays host or device; stream: cudaStream_t or NULL.  Returns
 * THC_ERR_NUMERIC if a normal-equation matrix stays singular after a ridge
 * of 1e-12 of its largest diagonal.  No context is needed.
 */
thc_status thc_cp_als(int n_occ, int n_vir, int n_rr, int rank, const double* U,
                      const double* eps, double* y_o, double* y_v, double* tau, int iters,
                      double* objective, void* stream);

/*
 * thc_selftest_gemm - randomised check of the tensor-core product (tcgen05,
 * bf16 hi/lo) against the CUDA-core product on the same float32 operands:
 * `cases` random shapes (M, N <= 700, K <= 900, batch <= 4), transposed and
 * plain operands, separate / shared / batch-reduced batches, split-K, beta
 * 0 or 0.5, three or one bf16 products.  *max_rel_err (nullable) = largest
 * bf16x3 difference relative to max(1, max|C|); *failures (nullable) =
 * cases outside the bound of their arithmetic (bf16x3: 2e-5 sqrt(K+1),
 * bf16: 2e-2 sqrt(K+1), times sqrt(batch) when batch-reduced).  Returns
 * THC_ERR_NUMERIC if any case fails.  Diagnostic; no counterpart in the paper.
 */
thc_status thc_selftest_gemm(int cases, unsigned long long seed, double* max_rel_err,
                             int* failures, void* stream);

/*
 * thc_selftest_gemm_f64 - randomised check of the float64 tensor-core
 * products (THC_PREC_FP64_TC) against the float64 CUDA-core products:
 * `cases` random shapes (up to three exact K chunks), orientations, batch
 * modes and beta, entries uniform or spread over 2^-40 .. 1.  *max_rel: the
 * largest max|difference| / max(1, max|C|); *failures: cases above
 * 1e-15 (K + 1).  Errors: THC_ERR_CUDA.
 */
thc_status thc_selftest_gemm_f64(int cases, unsigned long long seed, double* max_rel,
                                 int* failures, void* stream);

/*
 * thc_selftest_bounded_wait - exercise the bounded-wait path that every
 * waiting kernel of this library uses (TMA and MMA pipelines, the triangle
 * kernel's operand ring).  One thread waits on a shared-memory mbarrier that
 * is completed beforehand only if `complete` is non-zero, with a budget of
 * about a millisecond; on expiry the kernel raises a device flag and
 * returns, as the production kernels do, and this call reports it.
 * Returns THC_OK if the wait completed, THC_ERR_TIMEOUT if it expired (the
 * device stays usable either way), THC_ERR_CUDA on a launch failure.
 * stream: cudaStream_t or NULL.  No counterpart in the paper.
 */
thc_status thc_selftest_bounded_wait(int complete, void* stream);

/*
 * thc_probe_alu - measured CUDA-core FMA throughput of the current device
 * (the denominators of the triangle kernels' rooflines): `kind` 0 = float64
 * FMA, 1 = float32 FMA, 2 = packed float32 pairs (fma.rn.f32x2).  Eight
 * independent FMA chains per thread, 8 blocks of 256 threads per SM, one
 * timed launch after a warm-up (CUDA events on `stream`); *tflops counts
 * 2 flops per FMA lane.  Diagnostic; no counterpart in the paper.
 */
thc_status thc_probe_alu(int kind, double* tflops, void* stream);

/*
 * thc_probe_gemm - time of one tensor-core product C = A B (M x K times
 * K x N, row-major, seeded uniform operands in [-1, 1]) averaged over
 * `iters` products after two warm-up products, CUDA events on `stream`:
 *   mode 0  float32 operands, bf16 hi*hi + hi*lo + lo*hi, packed operands
 *           cached (the product kernel alone)
 *   mode 1  the same with the bf16 hi/lo pack of both operands in every call
 *   mode 2  bf16 hi*hi only, packed operands cached
 *   mode 3  float64 operands as exact integer slices (THC_PREC_FP64_TC):
 *           row exponents, slicing, 8 level products and the float64 pass
 * *ms = milliseconds per product.  Allocates its operands and workspace.
 * Errors: THC_ERR_ARG, THC_ERR_OOM, THC_ERR_CUDA, THC_ERR_TIMEOUT.
 * Diagnostic; no counterpart in the paper.
 */
thc_status thc_probe_gemm(int mode, int M, int N, int K, int iters, double* ms, void* stream);

/* Text of the first error recorded on ctx ("" if none).  The pointer stays
 * valid until the next call on ctx or thc_destroy.  ctx may be NULL, which
 * returns the last error of a failed thc_init, thc_energy_noalloc or
 * thc_probe_* call on this thread. */
const char* thc_last_error(const thc_ctx* ctx);

/* Release every device buffer of ctx.  NULL is accepted. */
void thc_destroy(thc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* THC_H */
