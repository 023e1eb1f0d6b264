// Learned preconditioner: a pointwise MLP over the elements of the working
// basis, with its own forward, backward and Adam kernels.
#pragma once

#include "common.cuh"
#include "gemm_tc.cuh"

namespace thc {

// Input features per element (P, Q) of the working basis (see mlp.cu).
constexpr int kMlpFeatures = 8;

template <typename T>
struct DBuf;

struct Mlp {
    int F = kMlpFeatures, H = 256;
    bool bf16 = true;            // bf16 weights/activations in the H x H layer
    long long np = 0;            // parameters
    cudaStream_t st = nullptr;
    int step = 0;                // Adam step count
    float* theta = nullptr;      // [W1 | b1 | W2 | b2 | w3 | b3]
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    // scratch for batches of up to cap samples
    long long cap = 0;
    float *a1 = nullptr, *a2 = nullptr, *d1 = nullptr, *d2 = nullptr;
    float *y = nullptr, *dy = nullptr, *ones = nullptr, *red = nullptr;
    float *xb = nullptr, *jb = nullptr, *tb = nullptr;
    float* splitk = nullptr;
    size_t splitk_elems = 0;
    TcWorkspace tc{};
    long long* perm = nullptr;

    Err create(int hidden, unsigned long long seed, bool use_bf16, cudaStream_t s);
    void destroy();
    Err ensure(long long n);
    // y[n] = net(X[n])  (X: n x F row-major, device)
    Err forward(const float* X, long long n, float* yout);
    // loss and gradient (into grad) of L = mean (j (1 + y) - t)^2
    Err loss_grad(const float* X, const float* j, const float* t, long long n, double* loss);
    Err adam(float lr);
    Err train(const float* X, const float* j, const float* t, long long n, int epochs,
              int batch, float lr, unsigned long long seed, double* final_loss);

    float* W1() const { return theta; }
    float* b1() const { return theta + (long long)H * F; }
    float* W2() const { return b1() + H; }
    float* b2() const { return W2() + (long long)H * H; }
    float* w3() const { return b2() + H; }
    float* b3() const { return w3() + H; }
};

// Features of the elements of the solver state x = [t1 (o v) | T (r r)] for
// one iteration (T in the working basis).
//   sig1 o x v  singles residual;  eps  o + v orbital energies
//   sq   r x r  projected residual C^T sigma C;   e  r  working-basis eigenvalues
//   x    state;  dprev  previous step (x_k - x_{k-1}), or null
//   idx  element indices into x, or null for all o v + r^2 elements
// X (n x F) features, jj (n) scaled Jacobi step; s1, s2 = RMS of the singles
// and doubles Jacobi steps.
cudaError_t mlp_features(const double* sig1, const double* eps, const double* sq,
                         const double* e, const double* x, const double* dprev,
                         const long long* idx, long long n, int o, int v, int r, double s1,
                         double s2, double log_rnorm, float* X, float* jj, cudaStream_t st);

// step[el] = (Jacobi step of el) * (1 + clamp(y[el], -0.95, 4)) for the
// elements of the blocks selected by `blocks` (bit 0 singles, bit 1
// doubles), the plain Jacobi step elsewhere.
cudaError_t mlp_apply(const double* sig1, const double* eps, const double* sq, const double* e,
                      const float* y, int o, int v, int r, int blocks, double* step,
                      cudaStream_t st);

}  // namespace thc
