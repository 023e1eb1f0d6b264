// Learned preconditioner network: forward, backward and Adam on the GPU.
//
// A pointwise MLP (F = 8 inputs, two tanh layers of width H, one output)
// maps features of a working-basis element (P, Q) to a factor on its Jacobi
// step: step = -sigma_q^PQ / (e_P + e_Q) * (1 + y).  The H x H layer runs on
// the tensor cores with bf16 weights and activations and float32
// accumulation (bf16 mode) or on the CUDA cores in float32; everything else
// is float32.  Loss for training samples (scaled Jacobi step j, scaled
// target step t):  L = mean_n (j_n (1 + y_n) - t_n)^2.
#include <cmath>
#include <vector>

#include "mlp.cuh"

namespace thc {
namespace {

constexpr int NT = 256;

unsigned nbl(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + NT - 1) / NT, 152 * 16)); }

__global__ void k_bias_tanh(float* Z, const float* b, long long n, int H) {
    const long long tot = n * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x)
        Z[i] = tanhf(Z[i] + b[i % H]);
}

__global__ void k_add_scalar(float* y, const float* b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] += b[0];
}

// dy = (2/n) (j (1 + y) - t) j ; part[block] = sum of r^2 (float64)
__global__ void k_loss(const float* y, const float* j, const float* t, long long n, float* dy,
                       double* part) {
    __shared__ double red[NT];
    double acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float r = j[i] * (1.f + y[i]) - t[i];
        dy[i] = (2.f / (float)n) * r * j[i];
        acc += (double)r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_d(const double* part, int n, double* out) {
    __shared__ double red[NT];
    double acc = 0;
    for (int i = threadIdx.x; i < n; i += NT) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// d2 = (dy w3^T) o (1 - a2^2)
__global__ void k_d2(const float* dy, const float* w3, const float* a2, long long n, int H,
                     float* d2) {
    const long long tot = n * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = a2[i];
        d2[i] = dy[i / H] * w3[i % H] * (1.f - a * a);
    }
}

__global__ void k_dtanh(float* d, const float* a, long long tot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = a[i];
        d[i] *= 1.f - x * x;
    }
}

__global__ void k_fill(float* p, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_adam(float* th, const float* g, float* m, float* v, long long n, float lr,
                       float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Minibatch gather through the pseudo-permutation i -> (off + i * stride) mod n.
__global__ void k_gather(const float* X, const float* j, const float* t, long long n, int F,
                         long long off, long long stride, long long b0, long long nb, float* xb,
                         float* jb, float* tb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
         i += (long long)gridDim.x * blockDim.x) {
        const long long src = (off + (b0 + i) % n * stride) % n;
        for (int f = 0; f < F; ++f) xb[i * F + f] = X[src * F + f];
        jb[i] = j[src];
        tb[i] = t[src];
    }
}

__device__ __forceinline__ float clipf(double x, double c) {
    return (float)fmin(c, fmax(-c, x));
}

// Element el of the state x = [t1 (o v) | T (r r)]: residual, denominator of
// its Jacobi step and the two orbital-like energies whose sum it is
// (singles (i, a): -eps_i and eps_a; doubles (P, Q): e_P and e_Q).
struct ElemView {
    double res, eP, eQ;
};

__device__ __forceinline__ ElemView elem(const double* sig1, const double* eps, const double* sq,
                                         const double* e, int o, int v, int r, long long el) {
    const long long ov = (long long)o * v;
    ElemView w;
    if (el < ov) {
        const int i = (int)(el / v), a = (int)(el % v);
        w.res = sig1[el];
        w.eP = -eps[i];
        w.eQ = eps[o + a];
    } else {
        const long long q = el - ov;
        const int p = (int)(q / r), qq = (int)(q % r);
        w.res = sq[q];
        w.eP = e[p];
        w.eQ = e[qq];
    }
    return w;
}

__global__ void k_features(const double* sig1, const double* eps, const double* sq,
                           const double* e, const double* x, const double* dprev,
                           const long long* idx, long long n, int o, int v, int r, double s1,
                           double s2, double logr, float* X, float* jj) {
    const long long ov = (long long)o * v;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long el = idx ? idx[k] : k;
        const ElemView w = elem(sig1, eps, sq, e, o, v, r, el);
        const bool singles = el < ov;
        const double s = singles ? s1 : s2;
        const double jac = -w.res / (w.eP + w.eQ);
        const double t = x[el] / s;
        float* f = X + k * kMlpFeatures;
        f[0] = (float)(0.5 * w.eP);
        f[1] = (float)(0.5 * w.eQ);
        f[2] = clipf(jac / s, 10.0);
        f[3] = dprev ? clipf(dprev[el] / s, 10.0) : 0.f;
        f[4] = (float)(copysign(log1p(fabs(t)), t) * 0.2);
        f[5] = (float)(0.1 * logr);
        f[6] = (float)(0.5 * fabs(w.eP - w.eQ));
        f[7] = singles ? -1.f : 1.f;
        jj[k] = (float)(jac / s);
    }
}

__global__ void k_apply(const double* sig1, const double* eps, const double* sq, const double* e,
                        const float* y, int o, int v, int r, int blocks, double* step) {
    const long long ov = (long long)o * v, tot = ov + (long long)r * r;
    for (long long el = blockIdx.x * (long long)blockDim.x + threadIdx.x; el < tot;
         el += (long long)gridDim.x * blockDim.x) {
        const ElemView w = elem(sig1, eps, sq, e, o, v, r, el);
        const bool on = (el < ov ? (blocks & 1) : (blocks & 2)) != 0;
        const double f = on ? 1.0 + fmin(4.0, fmax(-0.95, (double)y[el])) : 1.0;
        step[el] = -w.res / (w.eP + w.eQ) * f;
    }
}

unsigned long long splitmix(unsigned long long& s) {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

cudaError_t mlp_features(const double* sig1, const double* eps, const double* sq,
                         const double* e, const double* x, const double* dprev,
                         const long long* idx, long long n, int o, int v, int r, double s1,
                         double s2, double log_rnorm, float* X, float* jj, cudaStream_t st) {
    k_features<<<nbl(n), NT, 0, st>>>(sig1, eps, sq, e, x, dprev, idx, n, o, v, r, s1, s2,
                                      log_rnorm, X, jj);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_apply(const double* sig1, const double* eps, const double* sq, const double* e,
                      const float* y, int o, int v, int r, int blocks, double* step,
                      cudaStream_t st) {
    k_apply<<<nbl((long long)o * v + (long long)r * r), NT, 0, st>>>(sig1, eps, sq, e, y, o, v, r,
                                                                     blocks, step);
    count_launches(1);
    return cudaGetLastError();
}

Err Mlp::create(int hidden, unsigned long long seed, bool use_bf16, cudaStream_t s) {
    H = hidden;
    bf16 = use_bf16;
    st = s;
    np = (long long)H * F + H + (long long)H * H + H + H + 1;
    THC_CUDA(cudaMalloc(&theta, np * sizeof(float)));
    THC_CUDA(cudaMalloc(&grad, np * sizeof(float)));
    THC_CUDA(cudaMalloc(&m, np * sizeof(float)));
    THC_CUDA(cudaMalloc(&v, np * sizeof(float)));
    THC_CUDA(cudaMemsetAsync(m, 0, np * sizeof(float), st));
    THC_CUDA(cudaMemsetAsync(v, 0, np * sizeof(float), st));
    // Glorot-uniform hidden weights, zero biases and output layer: the
    // untrained network outputs 0, i.e. the plain Jacobi step.
    std::vector<float> h(np, 0.f);
    unsigned long long sd = seed;
    auto uni = [&]() { return (double)(splitmix(sd) >> 11) * (1.0 / 9007199254740992.0) * 2 - 1; };
    const double s1 = std::sqrt(6.0 / (F + H)), s2 = std::sqrt(6.0 / (2.0 * H));
    for (long long i = 0; i < (long long)H * F; ++i) h[i] = (float)(uni() * s1);
    float* w2 = h.data() + (long long)H * F + H;
    for (long long i = 0; i < (long long)H * H; ++i) w2[i] = (float)(uni() * s2);
    THC_CUDA(cudaMemcpy(theta, h.data(), np * sizeof(float), cudaMemcpyHostToDevice));
    step = 0;
    return Err{};
}

void Mlp::destroy() {
    for (float* p : {theta, grad, m, v, a1, a2, d1, d2, y, dy, ones, red, xb, jb, tb, splitk})
        if (p) cudaFree(p);
    if (tc.buf) cudaFree(tc.buf);
    if (tc.partial) cudaFree(tc.partial);
    if (tc.err) cudaFree(tc.err);
    theta = grad = m = v = a1 = a2 = d1 = d2 = y = dy = ones = red = xb = jb = tb = splitk = nullptr;
    tc = TcWorkspace{};
    cap = 0;
}

Err Mlp::ensure(long long n) {
    if (n <= cap) return Err{};
    for (float* p : {a1, a2, d1, d2, y, dy, ones, red, xb, jb, tb, splitk})
        if (p) cudaFree(p);
    if (tc.buf) cudaFree(tc.buf);
    if (tc.partial) cudaFree(tc.partial);
    if (tc.err) cudaFree(tc.err);
    cap = std::max<long long>(n, 4096);
    THC_CUDA(cudaMalloc(&a1, cap * H * sizeof(float)));
    THC_CUDA(cudaMalloc(&a2, cap * H * sizeof(float)));
    THC_CUDA(cudaMalloc(&d1, cap * H * sizeof(float)));
    THC_CUDA(cudaMalloc(&d2, cap * H * sizeof(float)));
    THC_CUDA(cudaMalloc(&y, cap * sizeof(float)));
    THC_CUDA(cudaMalloc(&dy, cap * sizeof(float)));
    THC_CUDA(cudaMalloc(&ones, cap * sizeof(float)));
    THC_CUDA(cudaMalloc(&red, 4096 * sizeof(double)));
    THC_CUDA(cudaMalloc(&xb, cap * F * sizeof(float)));
    THC_CUDA(cudaMalloc(&jb, cap * sizeof(float)));
    THC_CUDA(cudaMalloc(&tb, cap * sizeof(float)));
    splitk_elems = (size_t)std::max<long long>(64LL * H * H, 1 << 20);
    THC_CUDA(cudaMalloc(&splitk, splitk_elems * sizeof(float)));
    k_fill<<<nbl(cap), NT, 0, st>>>(ones, cap, 1.f);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    tc.elems = gemm_tc_pack_elems((int)std::min<long long>(cap, INT32_MAX), H, H, 1, false);
    THC_CUDA(cudaMalloc(&tc.buf, tc.elems * sizeof(__nv_bfloat16)));
    tc.partial_elems = (size_t)16 * H * H;
    THC_CUDA(cudaMalloc(&tc.partial, tc.partial_elems * sizeof(float)));
    THC_CUDA(cudaMalloc(&tc.err, sizeof(int)));
    THC_CUDA(cudaMemsetAsync(tc.err, 0, sizeof(int), st));
    return Err{};
}

static Err mm32(const Mlp& M, int Mr, int N, int K, View<float> A, View<float> B, float* C,
                long long ldc, double alpha, double beta) {
    Gemm<float> g;
    g.M = Mr; g.N = N; g.K = K; g.A = A; g.B = B; g.C = C; g.ldc = ldc;
    g.alpha = alpha; g.beta = beta;
    g.ws = M.splitk; g.ws_elems = M.splitk_elems;
    THC_CUDA(gemm_simt(g, M.st));
    return Err{};
}

Err Mlp::forward(const float* X, long long n, float* yout) {
    THC_TRY(ensure(n));
    const int ni = (int)n;
    // a1 = tanh(X W1^T + b1)
    THC_TRY(mm32(*this, ni, H, F, View<float>{X, F, 1}, View<float>{W1(), 1, F}, a1, H, 1, 0));
    k_bias_tanh<<<nbl(n * H), NT, 0, st>>>(a1, b1(), n, H);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    // a2 = tanh(a1 W2^T + b2)   (tensor cores, bf16 weights, in bf16 mode)
    bool done = false;
    if (bf16) {
        Gemm<float> g;
        g.M = ni; g.N = H; g.K = H;
        g.A = View<float>{a1, H, 1};
        g.B = View<float>{W2(), 1, H};
        g.C = a2; g.ldc = H;
        cudaError_t e = gemm_tc(g, tc, 1, st);
        if (e == cudaSuccess) done = true;
        else if (e != cudaErrorMemoryAllocation) THC_CUDA(e);
    }
    if (!done) THC_TRY(mm32(*this, ni, H, H, View<float>{a1, H, 1}, View<float>{W2(), 1, H}, a2, H, 1, 0));
    k_bias_tanh<<<nbl(n * H), NT, 0, st>>>(a2, b2(), n, H);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    // y = a2 w3 + b3
    THC_TRY(mm32(*this, ni, 1, H, View<float>{a2, H, 1}, View<float>{w3(), 1, 0}, yout, 1, 1, 0));
    k_add_scalar<<<nbl(n), NT, 0, st>>>(yout, b3(), n);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    return Err{};
}

Err Mlp::loss_grad(const float* X, const float* j, const float* t, long long n, double* loss) {
    // Scratch first: `y` below must already be the buffer forward() writes.
    THC_TRY(ensure(n));
    THC_TRY(forward(X, n, y));
    const int ni = (int)n;
    const unsigned nb = std::min<unsigned>(nbl(n), 1024);
    double* part = reinterpret_cast<double*>(red);
    k_loss<<<nb, NT, 0, st>>>(y, j, t, n, dy, part);
    k_sum_d<<<1, NT, 0, st>>>(part, (int)nb, part + 2048);
    count_launches(2);
    THC_CUDA(cudaGetLastError());
    float* gW1 = grad;
    float* gb1 = gW1 + (long long)H * F;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (long long)H * H;
    float* gw3 = gb2 + H;
    float* gb3 = gw3 + H;
    // output layer
    THC_TRY(mm32(*this, H, 1, ni, View<float>{a2, 1, H}, View<float>{dy, 1, 0}, gw3, 1, 1, 0));
    THC_TRY(mm32(*this, 1, 1, ni, View<float>{ones, 0, 1}, View<float>{dy, 1, 0}, gb3, 1, 1, 0));
    // second layer
    k_d2<<<nbl(n * H), NT, 0, st>>>(dy, w3(), a2, n, H, d2);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    THC_TRY(mm32(*this, H, H, ni, View<float>{d2, 1, H}, View<float>{a1, H, 1}, gW2, H, 1, 0));
    THC_TRY(mm32(*this, 1, H, ni, View<float>{ones, 0, 1}, View<float>{d2, H, 1}, gb2, H, 1, 0));
    // first layer
    THC_TRY(mm32(*this, ni, H, H, View<float>{d2, H, 1}, View<float>{W2(), H, 1}, d1, H, 1, 0));
    k_dtanh<<<nbl(n * H), NT, 0, st>>>(d1, a1, n * H);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    THC_TRY(mm32(*this, H, F, ni, View<float>{d1, 1, H}, View<float>{X, F, 1}, gW1, F, 1, 0));
    THC_TRY(mm32(*this, 1, H, ni, View<float>{ones, 0, 1}, View<float>{d1, H, 1}, gb1, H, 1, 0));
    if (loss) {
        double h = 0;
        THC_CUDA(cudaMemcpyAsync(&h, part + 2048, sizeof(double), cudaMemcpyDeviceToHost, st));
        THC_CUDA(cudaStreamSynchronize(st));
        *loss = h / (double)n;
    }
    return Err{};
}

Err Mlp::adam(float lr) {
    ++step;
    const float c1 = 1.f - std::pow(0.9f, (float)step), c2 = 1.f - std::pow(0.999f, (float)step);
    k_adam<<<nbl(np), NT, 0, st>>>(theta, grad, m, v, np, lr, c1, c2);
    count_launches(1);
    THC_CUDA(cudaGetLastError());
    return Err{};
}

Err Mlp::train(const float* X, const float* j, const float* t, long long n, int epochs, int batch,
               float lr, unsigned long long seed, double* final_loss) {
    if (n <= 0 || epochs <= 0) return Err{THC_ERR_ARG, "mlp train: empty data"};
    const long long B = std::max<long long>(1, std::min<long long>(batch > 0 ? batch : 4096, n));
    THC_TRY(ensure(B));
    unsigned long long sd = seed;
    double last = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        // pseudo-permutation: stride coprime with n
        long long stride = (long long)(splitmix(sd) % (unsigned long long)n) | 1;
        auto gcd = [](long long a, long long b) { while (b) { long long t2 = a % b; a = b; b = t2; } return a; };
        while (gcd(stride, n) != 1) stride += 2;
        const long long off = (long long)(splitmix(sd) % (unsigned long long)n);
        double acc = 0;
        long long cnt = 0;
        for (long long b0 = 0; b0 < n; b0 += B) {
            const long long nb = std::min(B, n - b0);
            k_gather<<<nbl(nb), NT, 0, st>>>(X, j, t, n, F, off, stride, b0, nb, xb, jb, tb);
            count_launches(1);
            THC_CUDA(cudaGetLastError());
            double l = 0;
            THC_TRY(loss_grad(xb, jb, tb, nb, &l));
            THC_TRY(adam(lr));
            acc += l * nb;
            cnt += nb;
        }
        last = acc / (double)cnt;
    }
    if (final_loss) *final_loss = last;
    return Err{};
}

}  // namespace thc
