// Solver of the projected amplitude equations (float64 throughout).
#pragma once

#include <vector>

#include "engine.cuh"
#include "mlp.cuh"

namespace thc {

// Orthonormal working basis of Eq. 22 and the Jacobi + DIIS iteration.
//
// S^WX = o^WX v^WX (Eq. 10 with tau = 1) and
// F^WX = sum_ia y_i^W y_a^W (eps_a - eps_i) y_i^X y_a^X are formed in float64;
// C solves F C = S C diag(e) with C^T S C = 1 on the range of S (eigenvalues
// of S below cutoff * max are dropped).  With U~ = (y o y) C semi-unitary
// (Eq. 12), the Fock part of the projected doubles Jacobian is exactly
// e_P + e_Q, which is the Jacobi denominator used here.
struct Solver {
    int P = 0, r = 0, o = 0, v = 0;
    long long len = 0;                 // o v + r r
    DBuf<double> C, e, Sd, SC;         // P x r, r, P x P, P x r
    DBuf<double> Zc, tmp, sq;          // P x P, P x r, r x r
    DBuf<double> x, xnew, step;        // state vectors [t1 | T]
    DBuf<double> hx, he;               // DIIS history (diis_n x len each)
    DBuf<double> red, dots;            // reduction scratch
    DBuf<double> epsd;                 // n orbital energies
    DBuf<double> ws;                   // split-K workspace
    std::vector<double> B;             // DIIS overlap matrix (host)
    int nhist = 0, head = 0;
    // Where the last plain Jacobi + DIIS run stopped (at max_iter): x holds
    // the next point, hx/he/B/nhist/head the DIIS history.
    bool resumable = false;
    int it_done = 0, m_done = 0;
    double e_prev_done = 0, last_norm_done = 0, rho_done = 1;

    // Learned-preconditioner state: previous iterate, saved point of the last
    // proposal, features and network outputs for all r^2 elements.
    DBuf<double> xprev, dprev, saved_x, saved_j, smlp;
    DBuf<float> feat, jjb, yb;
    // Recorded training pairs (features, scaled Jacobi step, scaled target).
    DBuf<float> recX, recJ, recT;
    DBuf<double> recTk, recS;
    DBuf<long long> recIdx;
    long long n_rec = 0, cap_rec = 0;

    template <typename T>
    Err setup(Engine<T>& eng, double cutoff);
    template <typename T>
    Err run(Engine<T>& eng, const thc_solve_opts& opts, double* Zc_io, double* t1_io,
            thc_report* rep, Mlp* mlp);
    // Checkpoint of a resumable run as one host blob (see thc_solve_state_save).
    size_t state_bytes() const;
    Err state_save(void* buf, size_t bytes, cudaStream_t st) const;
    Err state_load(const void* buf, size_t bytes, cudaStream_t st);
    // Copy out the pairs recorded by the last run (host or device pointers).
    Err pairs(float* X, float* j, float* t, long long max_n, long long* n_out,
              cudaStream_t st);

    Err mm(cudaStream_t st, int M, int N, int K, View<double> A, View<double> Bv, double* Cp,
           long long ldc, double alpha, double beta);
};

}  // namespace thc
