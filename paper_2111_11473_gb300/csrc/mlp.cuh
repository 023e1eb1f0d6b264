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

// Features of the working-basis elements for one solver iteration.
//   sq   r x r  projected residual C^T sigma C;   e  r  working-basis eigenvalues
//   Tq   r x r  current T;  dprev r x r  previous step (x_k - x_{k-1}), or null
//   idx  element indices (p * r + q) or null for all r^2 elements
// X (n x F) features, jj (n) scaled Jacobi step; s = RMS of the Jacobi step.
cudaError_t mlp_features(const double* sq, const double* e, const double* Tq,
                         const double* dprev, const long long* idx, long long n, int r,
                         double s, double log_rnorm, float* X, float* jj, cudaStream_t st);

// step[k] = -sq/(e_P + e_Q) * (1 + clamp(y)) for all r^2 elements.
cudaError_t mlp_apply(const double* sq, const double* e, const float* y, int r, double* step,
                      cudaStream_t st);

}  // namespace thc
