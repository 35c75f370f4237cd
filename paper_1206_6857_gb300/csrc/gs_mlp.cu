// Pair-selector network: batched inference, loss gradient and Adam training
// (the learned part of the traversal; not in the paper, which only has the
// rule of Fig. 6).  Softmax cross entropy with per-sample weights:
//   L = (1/n) sum_n s_n (logsumexp(o_n) - o_n[y_n]).
//
// Training works on tiles of kTile samples per CTA with every activation in
// shared memory: forward (A1 = Z W1 + b1, A2 = relu(A1) W2 + b2,
// O = relu(A2) W3 + b3), then backward through the same buffers; each CTA
// adds its tile's weight gradients into an FP64 gradient with one atomic per
// parameter.  Minibatches visit the samples in the order of a per-epoch
// affine permutation i -> (a i + b) mod n, gcd(a, n) = 1.
#include <math.h>
#include <string.h>

#include "gs_internal.h"
#include "gs_mlp.cuh"

namespace gs {

constexpr int kTile = 128;     // samples per CTA in the gradient kernel
constexpr int kMlpTB = 256;

__device__ __forceinline__ void load_params(const float *__restrict__ p, float *s) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) s[i] = p[i];
    __syncthreads();
}

__global__ void __launch_bounds__(kMlpTB) k_mlp_forward(const float *__restrict__ params, const float *__restrict__ x,
                                                       int64_t n, float *__restrict__ out) {
    __shared__ __align__(16) float w[kMlpParams + 3];
    load_params(params, w);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float xi[kMlpIn], o[kMlpOut];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) xi[k] = x[i * kMlpIn + k];
        mlp_infer(w, xi, o);
#pragma unroll
        for (int c = 0; c < kMlpOut; ++c) out[i * kMlpOut + c] = o[c];
    }
}

// per-feature sum and sum of squares (FP64) for the input normalisation
__global__ void k_feature_moments(const float *__restrict__ x, int64_t n, double *acc) {
    __shared__ double s[2 * kMlpIn];
    if (threadIdx.x < 2 * kMlpIn) s[threadIdx.x] = 0.0;
    __syncthreads();
    double a[kMlpIn], b[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) a[k] = b[k] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) {
            const double v = (double)x[i * kMlpIn + k];
            a[k] += v;
            b[k] += v * v;
        }
    }
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) {
        atomicAdd(&s[k], a[k]);
        atomicAdd(&s[kMlpIn + k], b[k]);
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMlpIn) atomicAdd(&acc[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_set_norm(float *params, const double *acc, int64_t n) {
    const int k = threadIdx.x;
    if (k >= kMlpIn) return;
    const double mean = acc[k] / (double)n;
    const double var = fmax(acc[kMlpIn + k] / (double)n - mean * mean, 0.0);
    params[kOffMu + k] = (float)mean;
    params[kOffSc + k] = (float)(1.0 / fmax(sqrt(var), 1e-3));
}

struct GradArgs {
    const float *params;
    const float *x;
    const int32_t *y;
    const float *s;        // per-sample weights (nullable: 1)
    int64_t n;             // samples in the data set
    int64_t start, count;  // this batch: permuted positions [start, start + count)
    uint64_t pa, pb;       // permutation i -> (pa i + pb) mod n
    double inv_count;      // 1 / count
    double *grad;          // kMlpParams, accumulated
    double *loss;          // accumulated batch loss
};

// Shared memory: params, Z[kTile][12], A1[kTile][64], A2[kTile][64],
// G[kTile][64], dO[kTile][5].
constexpr size_t kGradSmem =
    (size_t)(kMlpParams + 3 + kTile * (kMlpIn + 3 * kMlpHid + kMlpOut + 1)) * sizeof(float) + 64;

__global__ void __launch_bounds__(kMlpTB) k_mlp_grad(GradArgs ga) {
    extern __shared__ __align__(16) float sm[];
    float *w = sm;
    float *Z = w + kMlpParams + 3;
    float *A1 = Z + kTile * kMlpIn;
    float *A2 = A1 + kTile * kMlpHid;
    float *G = A2 + kTile * kMlpHid;
    float *dO = G + kTile * kMlpHid;
    float *Sw = dO + kTile * kMlpOut;
    load_params(ga.params, w);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t t0 = ga.start + (int64_t)blockIdx.x * kTile;
    const int nb = (int)min((int64_t)kTile, ga.start + ga.count - t0);
    if (nb <= 0) return;
    __shared__ int32_t ys[kTile];
    // inputs (normalised) of the tile
    for (int e = tid; e < nb * kMlpIn; e += nt) {
        const int m = e / kMlpIn, k = e % kMlpIn;
        const uint64_t pos = (uint64_t)(t0 + m);
        const int64_t src = (int64_t)((ga.pa * pos + ga.pb) % (uint64_t)ga.n);
        Z[m * kMlpIn + k] = (ga.x[src * kMlpIn + k] - w[kOffMu + k]) * w[kOffSc + k];
        if (k == 0) {
            ys[m] = ga.y[src];
            Sw[m] = ga.s ? ga.s[src] : 1.f;
        }
    }
    __syncthreads();
    // forward
    for (int e = tid; e < nb * kMlpHid; e += nt) {
        const int m = e / kMlpHid, i = e % kMlpHid;
        float a = w[kOffB1 + i];
        for (int k = 0; k < kMlpIn; ++k) a += Z[m * kMlpIn + k] * w[kOffW1 + k * kMlpHid + i];
        A1[e] = a;
    }
    __syncthreads();
    for (int e = tid; e < nb * kMlpHid; e += nt) {
        const int m = e / kMlpHid, j = e % kMlpHid;
        float a = w[kOffB2 + j];
        for (int i = 0; i < kMlpHid; ++i) a += relu_f(A1[m * kMlpHid + i]) * w[kOffW2 + i * kMlpHid + j];
        A2[e] = a;
    }
    __syncthreads();
    double lsum = 0.0;
    for (int m = tid; m < nb; m += nt) {
        float o[kMlpOut];
        for (int c = 0; c < kMlpOut; ++c) {
            float a = w[kOffB3 + c];
            for (int j = 0; j < kMlpHid; ++j) a += relu_f(A2[m * kMlpHid + j]) * w[kOffW3 + j * kMlpOut + c];
            o[c] = a;
        }
        float mx = o[0];
        for (int c = 1; c < kMlpOut; ++c) mx = fmaxf(mx, o[c]);
        float se = 0.f;
        for (int c = 0; c < kMlpOut; ++c) se += expf(o[c] - mx);
        const int y = ys[m];
        const float sw = Sw[m];
        lsum += (double)sw * ((double)mx + log((double)se) - (double)o[y]);
        const float scale = (float)((double)sw * ga.inv_count);
        for (int c = 0; c < kMlpOut; ++c) dO[m * kMlpOut + c] = scale * (expf(o[c] - mx) / se - (c == y ? 1.f : 0.f));
    }
    __syncthreads();
    // dW3, db3
    for (int e = tid; e < kMlpHid * kMlpOut + kMlpOut; e += nt) {
        double g = 0.0;
        if (e < kMlpHid * kMlpOut) {
            const int j = e / kMlpOut, c = e % kMlpOut;
            for (int m = 0; m < nb; ++m) g += (double)(relu_f(A2[m * kMlpHid + j]) * dO[m * kMlpOut + c]);
            atomicAdd(&ga.grad[kOffW3 + e], g);
        } else {
            const int c = e - kMlpHid * kMlpOut;
            for (int m = 0; m < nb; ++m) g += (double)dO[m * kMlpOut + c];
            atomicAdd(&ga.grad[kOffB3 + c], g);
        }
    }
    // G = dA2 = (dO W3^T) * [A2 > 0]
    for (int e = tid; e < nb * kMlpHid; e += nt) {
        const int m = e / kMlpHid, j = e % kMlpHid;
        float g = 0.f;
        for (int c = 0; c < kMlpOut; ++c) g += dO[m * kMlpOut + c] * w[kOffW3 + j * kMlpOut + c];
        G[e] = A2[e] > 0.f ? g : 0.f;
    }
    __syncthreads();
    // dW2, db2
    for (int e = tid; e < kMlpHid * kMlpHid + kMlpHid; e += nt) {
        double g = 0.0;
        if (e < kMlpHid * kMlpHid) {
            const int i = e / kMlpHid, j = e % kMlpHid;
            for (int m = 0; m < nb; ++m) g += (double)(relu_f(A1[m * kMlpHid + i]) * G[m * kMlpHid + j]);
            atomicAdd(&ga.grad[kOffW2 + e], g);
        } else {
            const int j = e - kMlpHid * kMlpHid;
            for (int m = 0; m < nb; ++m) g += (double)G[m * kMlpHid + j];
            atomicAdd(&ga.grad[kOffB2 + j], g);
        }
    }
    // dA1 = (G W2^T) * [A1 > 0], into A2 (no longer needed)
    for (int e = tid; e < nb * kMlpHid; e += nt) {
        const int m = e / kMlpHid, i = e % kMlpHid;
        float g = 0.f;
        for (int j = 0; j < kMlpHid; ++j) g += G[m * kMlpHid + j] * w[kOffW2 + i * kMlpHid + j];
        A2[e] = A1[e] > 0.f ? g : 0.f;
    }
    __syncthreads();
    // dW1, db1
    for (int e = tid; e < kMlpIn * kMlpHid + kMlpHid; e += nt) {
        double g = 0.0;
        if (e < kMlpIn * kMlpHid) {
            const int k = e / kMlpHid, i = e % kMlpHid;
            for (int m = 0; m < nb; ++m) g += (double)(Z[m * kMlpIn + k] * A2[m * kMlpHid + i]);
            atomicAdd(&ga.grad[kOffW1 + e], g);
        } else {
            const int i = e - kMlpIn * kMlpHid;
            for (int m = 0; m < nb; ++m) g += (double)A2[m * kMlpHid + i];
            atomicAdd(&ga.grad[kOffB1 + i], g);
        }
    }
    // batch loss
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0 && lsum != 0.0) atomicAdd(ga.loss, lsum * ga.inv_count);
}

// Adam on the trained entries (everything after mu and sc); t is the step (>= 1)
__global__ void k_mlp_adam(float *params, const double *grad, float *m, float *v, int t, float lr) {
    const int i = kOffW1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float g = (float)grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    params[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

static uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint64_t gcd_u64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static int launch_grad(const float *params, const float *x, const int32_t *y, const float *s, int64_t n,
                       int64_t start, int64_t count, uint64_t pa, uint64_t pb, double *grad, double *loss,
                       cudaStream_t st) {
    GradArgs ga;
    ga.params = params; ga.x = x; ga.y = y; ga.s = s; ga.n = n;
    ga.start = start; ga.count = count; ga.pa = pa; ga.pb = pb;
    ga.inv_count = 1.0 / (double)count;
    ga.grad = grad; ga.loss = loss;
    GS_CUDA_TRY(allow_max_smem((const void *)k_mlp_grad));
    const unsigned grid = (unsigned)((count + kTile - 1) / kTile);
    k_mlp_grad<<<grid, kMlpTB, kGradSmem, st>>>(ga);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_mlp_forward(const float *params, const float *x, int64_t n, float *logits, void *stream) {
    if (!params || (n > 0 && (!x || !logits)) || n < 0) {
        set_error("gs_mlp_forward: null pointer or negative n");
        return GS_ERR_ARG;
    }
    if (n == 0) return GS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t g = (n + kMlpTB - 1) / kMlpTB;
    k_mlp_forward<<<(unsigned)(g < 4096 ? g : 4096), kMlpTB, 0, st>>>(params, x, n, logits);
    GS_CUDA_TRY(cudaGetLastError());
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    return GS_OK;
}

extern "C" int gs_mlp_loss_grad(const float *params, const float *x, const int32_t *y, const float *s, int64_t n,
                                double *grad, double *loss, void *stream) {
    if (!params || !x || !y || !grad || !loss || n <= 0) {
        set_error("gs_mlp_loss_grad: null pointer or n <= 0");
        return GS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(double), st));
    GS_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), st));
    if (int rc = launch_grad(params, x, y, s, n, 0, n, 1, 0, grad, loss, st)) return rc;
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    return GS_OK;
}

extern "C" int gs_mlp_train(float *params, const float *x, const int32_t *y, const float *s, int64_t n, int epochs,
                            int batch, double lr, uint64_t seed, int set_norm, double *epoch_loss, void *stream) {
    if (!params || !x || !y || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.0)) {
        set_error("gs_mlp_train: bad arguments");
        return GS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double *grad = nullptr, *loss = nullptr, *acc = nullptr;
    float *m = nullptr, *v = nullptr;
    int rc = GS_OK;
    auto fail = [&](cudaError_t e, const char *what) { rc = cuda_fail(e, what); };
    cudaError_t e = dev_malloc_async((void **)&grad, kMlpParams * sizeof(double), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&loss, (size_t)(epochs + 1) * sizeof(double), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&acc, 2 * kMlpIn * sizeof(double), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&m, 2 * kMlpParams * sizeof(float), st);
    if (e != cudaSuccess) {
        fail(e, "gs_mlp_train scratch");
    } else {
        v = m + kMlpParams;
        cudaMemsetAsync(m, 0, 2 * kMlpParams * sizeof(float), st);
        cudaMemsetAsync(loss, 0, (size_t)(epochs + 1) * sizeof(double), st);
        if (set_norm) {
            cudaMemsetAsync(acc, 0, 2 * kMlpIn * sizeof(double), st);
            const int64_t g = (n + kMlpTB - 1) / kMlpTB;
            k_feature_moments<<<(unsigned)(g < 1024 ? g : 1024), kMlpTB, 0, st>>>(x, n, acc);
            k_set_norm<<<1, 32, 0, st>>>(params, acc, n);
        }
        uint64_t rs = seed;
        int t = 0;
        for (int ep = 0; ep < epochs && rc == GS_OK; ++ep) {
            uint64_t pa = 1, pb = 0;
            if (n > 1) {
                do { pa = 1 + splitmix64(rs) % (uint64_t)(n - 1); } while (gcd_u64(pa, (uint64_t)n) != 1);
                pb = splitmix64(rs) % (uint64_t)n;
            }
            for (int64_t s0 = 0; s0 < n && rc == GS_OK; s0 += batch) {
                const int64_t cnt = (n - s0) < batch ? (n - s0) : batch;
                cudaMemsetAsync(grad, 0, kMlpParams * sizeof(double), st);
                rc = launch_grad(params, x, y, s, n, s0, cnt, pa, pb, grad, loss + ep, st);
                if (rc) break;
                ++t;
                k_mlp_adam<<<(kMlpParams - kOffW1 + 255) / 256, 256, 0, st>>>(params, grad, m, v, t, (float)lr);
                e = cudaGetLastError();
                if (e != cudaSuccess) fail(e, "k_mlp_adam");
            }
        }
        if (rc == GS_OK && epoch_loss && epochs > 0) {
            e = cudaMemcpyAsync(epoch_loss, loss, epochs * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) fail(e, "epoch losses");
        }
        e = cudaStreamSynchronize(st);
        if (rc == GS_OK && e != cudaSuccess) fail(e, "gs_mlp_train");
        if (rc == GS_OK && epoch_loss) {
            // per-epoch mean of the batch losses
            const int64_t nbat = (n + batch - 1) / batch;
            for (int ep = 0; ep < epochs; ++ep) epoch_loss[ep] /= (double)nbat;
        }
    }
    if (grad) cudaFreeAsync(grad, st);
    if (loss) cudaFreeAsync(loss, st);
    if (acc) cudaFreeAsync(acc, st);
    if (m) cudaFreeAsync(m, st);
    return rc;
}
