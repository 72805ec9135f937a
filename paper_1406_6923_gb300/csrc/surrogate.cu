// Learned surrogate of the offline stage (an extension of Algorithm 1 stage
// 1: when the velocity model changes between inversion iterations, a
// network maps each subdomain's velocity block to its S-fraction
// coefficients instead of the Krylov/Lanczos build of Eqs. 5-13).
//
// Network (FP32 training, BF16 or FP32 inference), all kernels written here:
//   input  log(c / c_ref) on the block's n^3 cells, one channel;
//   three 3x3x3 convolutions of stride 2, zero padding 1, ReLU
//   (n -> n/2 -> n/4 -> n/8 per axis);
//   a two-layer MLP (ReLU between) to a code z of dimension d.
// Decoder (FP64, fixed, not trained): r = mu + P z, mu and P the mean and a
// basis of the leading principal subspace of the training targets (found by
// randomized subspace iteration), r -> for every block Gamma_j, Gammahat_j
// (j >= 2) a factor L = U diag(exp(g)), U unit lower triangular, so each
// decoded block L L^T is positive definite whatever the network outputs.
// Level 1 comes from its closed forms in the builder (Gammahat_1 = F^T F,
// Gamma_1 = Gammahat_1^{-1} F^T L F Gammahat_1^{-1}).
// Judge: the NtD map S(lambda) = F^T (L + lambda)^{-1} F of the S-fraction
// (Eq. 15), evaluated by the continued fraction
//   Y_k = lambda Gammahat_k^{-1} + Gamma_k,
//   Y_j = lambda Gammahat_j^{-1} + (Gamma_j^{-1} + Y_{j+1}^{-1})^{-1},
//   S = Y_1^{-1},
// at complex lambda; the fallback compares S(sigma) with one block solve.
#include "sfm_internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace sfm {
namespace sur {

template <typename T>
__device__ __forceinline__ float ldf(const T* p) { return (float)*p; }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <typename T>
__device__ __forceinline__ void stf(T* p, float v) { *p = (T)v; }
template <>
__device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16(v); }

// x[s][i] = log(c[s][i] / c_ref)
template <typename T>
__global__ void features_kernel(const float* c, float c_ref, long long n, T* x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        stf(x + i, logf(c[i] / c_ref));
}

// a = conv(x, W) + b (stride 2, zero padding 1), h = relu(a) (h may be NULL).
// x [B][cin][n][n][n], W [cout][cin][3][3][3], a/h [B][cout][m][m][m].
template <typename T, typename TW>
__global__ void conv_fwd_kernel(const T* x, const TW* W, const TW* bias, int B, int cin, int n,
                                int cout, int m, float* a, T* h) {
    const long long total = (long long)B * cout * m * m * m;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const int ox = (int)(o % m), oy = (int)((o / m) % m), oz = (int)((o / ((long long)m * m)) % m);
        const int co = (int)((o / ((long long)m * m * m)) % cout);
        const int bt = (int)(o / ((long long)m * m * m * cout));
        float acc = ldf(bias + co);
        for (int ci = 0; ci < cin; ++ci) {
            const T* xc = x + ((long long)bt * cin + ci) * n * n * n;
            const TW* w = W + ((long long)co * cin + ci) * 27;
            for (int dz = 0; dz < 3; ++dz) {
                const int iz = 2 * oz + dz - 1;
                if (iz < 0 || iz >= n) continue;
                for (int dy = 0; dy < 3; ++dy) {
                    const int iy = 2 * oy + dy - 1;
                    if (iy < 0 || iy >= n) continue;
                    for (int dx = 0; dx < 3; ++dx) {
                        const int ix = 2 * ox + dx - 1;
                        if (ix < 0 || ix >= n) continue;
                        acc = fmaf(ldf(w + (dz * 3 + dy) * 3 + dx), ldf(xc + ((long long)iz * n + iy) * n + ix), acc);
                    }
                }
            }
        }
        if (a) a[o] = acc;
        if (h) stf(h + o, fmaxf(acc, 0.f));
    }
}

// dx = conv^T(da, W): every input cell gathers the outputs that read it.
__global__ void conv_bwd_data_kernel(const float* da, const float* W, int B, int cin, int n, int cout,
                                     int m, float* dx) {
    const long long total = (long long)B * cin * n * n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)((i / ((long long)n * n)) % n);
        const int ci = (int)((i / ((long long)n * n * n)) % cin);
        const int bt = (int)(i / ((long long)n * n * n * cin));
        float acc = 0.f;
        for (int dz = 0; dz < 3; ++dz) {
            const int tz = iz + 1 - dz;
            if (tz < 0 || (tz & 1) || (tz >> 1) >= m) continue;
            for (int dy = 0; dy < 3; ++dy) {
                const int ty = iy + 1 - dy;
                if (ty < 0 || (ty & 1) || (ty >> 1) >= m) continue;
                for (int dx3 = 0; dx3 < 3; ++dx3) {
                    const int tx = ix + 1 - dx3;
                    if (tx < 0 || (tx & 1) || (tx >> 1) >= m) continue;
                    const long long op = ((long long)(tz >> 1) * m + (ty >> 1)) * m + (tx >> 1);
                    for (int co = 0; co < cout; ++co)
                        acc = fmaf(W[((long long)co * cin + ci) * 27 + (dz * 3 + dy) * 3 + dx3],
                                   da[((long long)bt * cout + co) * m * m * m + op], acc);
                }
            }
        }
        dx[i] = acc;
    }
}

// dW[co][ci][t] = sum over samples and output cells of da . x (one block per
// weight, fixed-order tree reduction); db[co] likewise from da alone.
__global__ void conv_bwd_w_kernel(const float* da, const float* x, int B, int cin, int n, int cout,
                                  int m, float* dW, float* db) {
    __shared__ float red[256];
    const int wid = blockIdx.x;                 // co * (cin * 27 + 1) + rest
    const int per = cin * 27 + 1;
    const int co = wid / per, r = wid - co * per;
    const long long cells = (long long)m * m * m;
    float acc = 0.f;
    if (r == cin * 27) {
        for (long long e = threadIdx.x; e < (long long)B * cells; e += blockDim.x) {
            const int bt = (int)(e / cells);
            acc += da[((long long)bt * cout + co) * cells + (e - bt * cells)];
        }
    } else {
        const int ci = r / 27, t = r % 27, dz = t / 9, dy = (t / 3) % 3, dx3 = t % 3;
        for (long long e = threadIdx.x; e < (long long)B * cells; e += blockDim.x) {
            const int bt = (int)(e / cells);
            const long long op = e - bt * cells;
            const int ox = (int)(op % m), oy = (int)((op / m) % m), oz = (int)(op / ((long long)m * m));
            const int iz = 2 * oz + dz - 1, iy = 2 * oy + dy - 1, ix = 2 * ox + dx3 - 1;
            if (iz < 0 || iz >= n || iy < 0 || iy >= n || ix < 0 || ix >= n) continue;
            acc = fmaf(da[((long long)bt * cout + co) * cells + op],
                       x[(((long long)bt * cin + ci) * n + iz) * n * n + (long long)iy * n + ix], acc);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (r == cin * 27) db[co] = red[0];
        else dW[(long long)co * cin * 27 + r] = red[0];
    }
}

// C[M][N] = alpha * op(A) op(B) + (beta ? C : 0) + bias[n] (optional), then
// relu (optional, also writing the pre-activation to Cpre when not NULL).
// op(A)[m][k] = TA ? A[k][m] : A[m][k] (lda its row length), likewise B.
// 16x16 output tiles, 16-deep K slabs in shared memory; the K sum runs in
// one fixed order, so the result does not depend on the launch.
template <typename T, typename TA_, typename TB_, bool TA, bool TB>
__global__ void gemm_kernel(int M, int N, int K, T alpha, const TA_* A, int lda, const TB_* B,
                            int ldb, T beta, T* C, int ldc, const TB_* bias, int relu, T* Cpre) {
    __shared__ T As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    T acc = T(0);
    for (int k0 = 0; k0 < K; k0 += 16) {
        {
            const int m = blockIdx.y * 16 + ty, k = k0 + tx;
            T v = T(0);
            if (m < M && k < K) v = (T)(TA ? ldf(A + (long long)k * lda + m) : ldf(A + (long long)m * lda + k));
            As[ty][tx] = v;
        }
        {
            const int k = k0 + ty, n = blockIdx.x * 16 + tx;
            T v = T(0);
            if (k < K && n < N) v = (T)(TB ? ldf(B + (long long)n * ldb + k) : ldf(B + (long long)k * ldb + n));
            Bs[ty][tx] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
        __syncthreads();
    }
    if (row < M && col < N) {
        T v = alpha * acc;
        if (beta != T(0)) v += beta * C[(long long)row * ldc + col];
        if (bias) v += (T)ldf(bias + col);
        if (Cpre) Cpre[(long long)row * ldc + col] = v;
        if (relu) v = v > T(0) ? v : T(0);
        C[(long long)row * ldc + col] = v;
    }
}

template <bool TA, bool TB>
__global__ void dgemm_kernel(int M, int N, int K, double alpha, const double* A, int lda, const double* B,
                             int ldb, double beta, double* C, int ldc) {
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        {
            const int m = blockIdx.y * 16 + ty, k = k0 + tx;
            As[ty][tx] = (m < M && k < K) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.0;
        }
        {
            const int k = k0 + ty, n = blockIdx.x * 16 + tx;
            Bs[ty][tx] = (k < K && n < N) ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (row < M && col < N) {
        double v = alpha * acc;
        if (beta != 0.0) v += beta * C[(long long)row * ldc + col];
        C[(long long)row * ldc + col] = v;
    }
}

// bias gradient of a dense layer: db[o] = sum over rows of dY[row][o]
__global__ void colsum_kernel(const float* dY, int rows, int cols, float* db) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dY[(long long)r * cols + o];
    db[o] = s;
}

// da = dh * (a > 0)
__global__ void relu_bwd_kernel(const float* dh, const float* a, long long n, float* da) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        da[i] = a[i] > 0.f ? dh[i] : 0.f;
}

// loss = mean over samples of mean over the code of (z - zt)^2, and its
// gradient dz = 2 (z - zt) / (d B); one block, fixed-order reduction
__global__ void mse_kernel(const float* z, const float* zt, int B, int d, float* dz, float* loss) {
    __shared__ float red[256];
    float acc = 0.f;
    const float sc = 1.f / ((float)d * (float)B);
    for (int i = threadIdx.x; i < B * d; i += blockDim.x) {
        const float e = z[i] - zt[i];
        acc += e * e;
        dz[i] = 2.f * e * sc;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] * sc;
}

// one Adam step (Kingma and Ba) on every parameter
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float mi = b1 * m[i] + (1.f - b1) * g[i];
        const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void to_bf16_kernel(const float* in, __nv_bfloat16* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(in[i]);
}

inline int grid1(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, 16384));
}

template <typename T, typename TA_, typename TB_, bool TA, bool TB>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, T alpha, const TA_* A, int lda, const TB_* B,
                 int ldb, T beta, T* C, int ldc, const TB_* bias = nullptr, int relu = 0,
                 T* Cpre = nullptr) {
    dim3 grid((N + 15) / 16, (M + 15) / 16);
    gemm_kernel<T, TA_, TB_, TA, TB><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                          bias, relu, Cpre);
    return cudaGetLastError();
}

template <bool TA, bool TB>
cudaError_t dgemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, int lda,
                  const double* B, int ldb, double beta, double* C, int ldc) {
    dim3 grid((N + 15) / 16, (M + 15) / 16);
    dgemm_kernel<TA, TB><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

}  // namespace sur
}  // namespace sfm


// ---------------------------------------------------------------------------
// The network object (opaque in the C ABI)
// ---------------------------------------------------------------------------

struct sfm_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int n = 24, c[3] = {16, 32, 64}, m[4] = {24, 12, 6, 3}, hidden = 1024, code = 64, flat = 0;
    long long off[11] = {0};       // parameter offsets: c1w c1b c2w c2b c3w c3b W1 b1 W2 b2 | end
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    __nv_bfloat16* pb = nullptr;   // BF16 copy of the parameters (inference)
    bool pb_valid = false;
    int t = 0;                     // Adam steps taken
    int cap = 0;                   // batch capacity of the activations
    float *x = nullptr, *a1 = nullptr, *h1 = nullptr, *a2 = nullptr, *h2 = nullptr, *a3 = nullptr,
          *h3 = nullptr, *amlp = nullptr, *hmlp = nullptr, *z = nullptr, *dz = nullptr, *t1 = nullptr,
          *t2 = nullptr, *loss = nullptr;
    __nv_bfloat16 *xb = nullptr, *h1b = nullptr, *h2b = nullptr, *h3b = nullptr;
    // decoder (FP64): raw = mu + P z, for blocks of width b and k levels
    int b = 0, k = 0, nraw = 0;
    double *mu = nullptr, *P = nullptr;
};

namespace {

using namespace sfm::sur;

int nfail(sfm_net* net, int code, const std::string& msg) {
    if (net) net->err = msg;
    else sfm::set_global_error(msg);
    return code;
}

#define NCK(net, call)                                                                          \
    do {                                                                                        \
        cudaError_t e__ = (call);                                                               \
        if (e__ != cudaSuccess)                                                                 \
            return nfail((net), e__ == cudaErrorMemoryAllocation ? SFM_ERR_NOMEM : SFM_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e__));                  \
    } while (0)

template <typename T>
void nfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

template <typename T>
cudaError_t nalloc(T*& p, size_t count) {
    nfree(p);
    return cudaMalloc((void**)&p, std::max<size_t>(count, 1) * sizeof(T));
}

void free_acts(sfm_net* net) {
    for (float** p : {&net->x, &net->a1, &net->h1, &net->a2, &net->h2, &net->a3, &net->h3, &net->amlp,
                      &net->hmlp, &net->z, &net->dz, &net->t1, &net->t2, &net->loss})
        nfree(*p);
    for (__nv_bfloat16** p : {&net->xb, &net->h1b, &net->h2b, &net->h3b}) nfree(*p);
    net->cap = 0;
}

// activations for a batch of B samples
int ensure_acts(sfm_net* net, int B) {
    if (B <= net->cap) return SFM_OK;
    free_acts(net);
    const long long n3 = (long long)net->n * net->n * net->n;
    long long s[4] = {n3, 0, 0, 0};
    for (int l = 1; l <= 3; ++l) s[l] = (long long)net->c[l - 1] * net->m[l] * net->m[l] * net->m[l];
    const long long big = std::max({n3, s[1], s[2], s[3], (long long)net->hidden});
    NCK(net, nalloc(net->x, B * n3));
    NCK(net, nalloc(net->a1, B * s[1]));
    NCK(net, nalloc(net->h1, B * s[1]));
    NCK(net, nalloc(net->a2, B * s[2]));
    NCK(net, nalloc(net->h2, B * s[2]));
    NCK(net, nalloc(net->a3, B * s[3]));
    NCK(net, nalloc(net->h3, B * s[3]));
    NCK(net, nalloc(net->amlp, (size_t)B * net->hidden));
    NCK(net, nalloc(net->hmlp, (size_t)B * net->hidden));
    NCK(net, nalloc(net->z, (size_t)B * net->code));
    NCK(net, nalloc(net->dz, (size_t)B * net->code));
    NCK(net, nalloc(net->t1, B * big));
    NCK(net, nalloc(net->t2, B * big));
    NCK(net, nalloc(net->xb, B * n3));
    NCK(net, nalloc(net->h1b, B * s[1]));
    NCK(net, nalloc(net->h2b, B * s[2]));
    NCK(net, nalloc(net->h3b, B * s[3]));
    NCK(net, nalloc(net->loss, 1));
    net->cap = B;
    return SFM_OK;
}

}  // namespace

extern "C" int sfm_net_create(sfm_net** out, int device, int n, int c1, int c2, int c3, int hidden,
                              int code, unsigned long long seed) {
    if (!out) return nfail(nullptr, SFM_ERR_ARG, "sfm_net_create: NULL output");
    *out = nullptr;
    if (n < 2 || c1 < 1 || c2 < 1 || c3 < 1 || hidden < 1 || code < 1)
        return nfail(nullptr, SFM_ERR_ARG, "sfm_net_create: bad sizes");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return nfail(nullptr, SFM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    sfm_net* net = new sfm_net();
    net->device = device;
    net->n = n;
    net->c[0] = c1; net->c[1] = c2; net->c[2] = c3;
    net->m[0] = n;
    for (int l = 1; l <= 3; ++l) net->m[l] = (net->m[l - 1] - 1) / 2 + 1;
    net->hidden = hidden;
    net->code = code;
    net->flat = c3 * net->m[3] * net->m[3] * net->m[3];
    const long long sizes[10] = {(long long)c1 * 27, c1, (long long)c2 * c1 * 27, c2, (long long)c3 * c2 * 27, c3,
                                 (long long)hidden * net->flat, hidden, (long long)code * hidden, code};
    net->off[0] = 0;
    for (int i = 0; i < 10; ++i) net->off[i + 1] = net->off[i] + sizes[i];
    const long long np = net->off[10];
    // He-style initialisation (seeded): conv and first dense weights with
    // variance 2 / fan_in, the last layer with 1 / fan_in, biases zero
    std::vector<float> w(np, 0.f);
    unsigned long long st = seed * 0x9e3779b97f4a7c15ull + 1;
    auto uni = [&]() {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    auto gauss = [&]() { return std::sqrt(-2.0 * std::log(uni())) * std::cos(6.283185307179586 * uni()); };
    const double fan[5] = {27.0, 27.0 * c1, 27.0 * c2, (double)net->flat, (double)hidden};
    const int widx[5] = {0, 2, 4, 6, 8};
    for (int l = 0; l < 5; ++l) {
        const double sd = std::sqrt((l == 4 ? 1.0 : 2.0) / fan[l]);
        for (long long i = net->off[widx[l]]; i < net->off[widx[l] + 1]; ++i) w[i] = (float)(sd * gauss());
    }
    int rc = SFM_OK;
    if ((e = cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = nalloc(net->params, np)) != cudaSuccess || (e = nalloc(net->grads, np)) != cudaSuccess ||
        (e = nalloc(net->am, np)) != cudaSuccess || (e = nalloc(net->av, np)) != cudaSuccess ||
        (e = nalloc(net->pb, np)) != cudaSuccess ||
        (e = cudaMemcpy(net->params, w.data(), np * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(net->am, 0, np * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(net->av, 0, np * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(net->grads, 0, np * sizeof(float))) != cudaSuccess)
        rc = nfail(nullptr, SFM_ERR_CUDA, std::string("sfm_net_create: ") + cudaGetErrorString(e));
    if (rc != SFM_OK) { sfm_net_destroy(net); return rc; }
    *out = net;
    return SFM_OK;
}

extern "C" int sfm_net_destroy(sfm_net* net) {
    if (!net) return SFM_OK;
    cudaSetDevice(net->device);
    if (net->stream) cudaStreamSynchronize(net->stream);
    free_acts(net);
    for (float** p : {&net->params, &net->grads, &net->am, &net->av}) nfree(*p);
    nfree(net->pb);
    nfree(net->mu);
    nfree(net->P);
    if (net->stream) cudaStreamDestroy(net->stream);
    delete net;
    return SFM_OK;
}

extern "C" const char* sfm_net_last_error(const sfm_net* net) { return net ? net->err.c_str() : ""; }

extern "C" int sfm_net_params(sfm_net* net, float* host, size_t capacity, size_t* count, int set) {
    if (!net) return nfail(nullptr, SFM_ERR_ARG, "NULL network");
    const size_t np = (size_t)net->off[10];
    if (count) *count = np;
    if (!host) return SFM_OK;
    if (capacity < np) return nfail(net, SFM_ERR_ARG, "sfm_net_params: capacity below the parameter count");
    NCK(net, cudaSetDevice(net->device));
    if (set) {
        NCK(net, cudaMemcpy(net->params, host, np * sizeof(float), cudaMemcpyHostToDevice));
        NCK(net, cudaMemset(net->am, 0, np * sizeof(float)));
        NCK(net, cudaMemset(net->av, 0, np * sizeof(float)));
        net->t = 0;
        net->pb_valid = false;
    } else {
        NCK(net, cudaMemcpy(host, net->params, np * sizeof(float), cudaMemcpyDeviceToHost));
    }
    return SFM_OK;
}

namespace {

// FP32 forward pass of a batch (training form: keeps the pre-activations)
int forward_f32(sfm_net* net, const float* c, int B) {
    cudaStream_t st = net->stream;
    const float* P = net->params;
    const long long n3 = (long long)net->n * net->n * net->n;
    features_kernel<float><<<grid1(B * n3), 256, 0, st>>>(c, 2500.f, B * n3, net->x);
    const float* in = net->x;
    float* as[3] = {net->a1, net->a2, net->a3};
    float* hs[3] = {net->h1, net->h2, net->h3};
    int cin = 1;
    for (int l = 0; l < 3; ++l) {
        const long long cells = (long long)B * net->c[l] * net->m[l + 1] * net->m[l + 1] * net->m[l + 1];
        conv_fwd_kernel<float, float><<<grid1(cells), 256, 0, st>>>(
            in, P + net->off[2 * l], P + net->off[2 * l + 1], B, cin, net->m[l], net->c[l], net->m[l + 1],
            as[l], hs[l]);
        in = hs[l];
        cin = net->c[l];
    }
    NCK(net, cudaGetLastError());
    NCK(net, (gemm<float, float, float, false, true>(st, B, net->hidden, net->flat, 1.f, net->h3, net->flat,
                                                    P + net->off[6], net->flat, 0.f, net->hmlp, net->hidden,
                                                    P + net->off[7], 1, net->amlp)));
    NCK(net, (gemm<float, float, float, false, true>(st, B, net->code, net->hidden, 1.f, net->hmlp,
                                                    net->hidden, P + net->off[8], net->hidden, 0.f, net->z,
                                                    net->code, P + net->off[9], 0, nullptr)));
    return SFM_OK;
}

}  // namespace

// Loss of a batch (mean squared code error) and the gradient of every
// parameter by the backward pass, left in the network for sfm_net_adam.
extern "C" int sfm_net_grad(sfm_net* net, const float* c, const float* zt, int B, float* loss,
                            float* grad_host) {
    if (!net || !c || !zt || B < 1) return nfail(net, SFM_ERR_ARG, "sfm_net_grad: bad arguments");
    NCK(net, cudaSetDevice(net->device));
    int rc = ensure_acts(net, B);
    if (rc) return rc;
    rc = forward_f32(net, c, B);
    if (rc) return rc;
    cudaStream_t st = net->stream;
    const float* P = net->params;
    float* G = net->grads;
    mse_kernel<<<1, 256, 0, st>>>(net->z, zt, B, net->code, net->dz, net->loss);
    // second dense layer
    NCK(net, (gemm<float, float, float, true, false>(st, net->code, net->hidden, B, 1.f, net->dz, net->code,
                                                    net->hmlp, net->hidden, 0.f, G + net->off[8], net->hidden)));
    colsum_kernel<<<(net->code + 127) / 128, 128, 0, st>>>(net->dz, B, net->code, G + net->off[9]);
    NCK(net, (gemm<float, float, float, false, false>(st, B, net->hidden, net->code, 1.f, net->dz, net->code,
                                                     P + net->off[8], net->hidden, 0.f, net->t1, net->hidden)));
    relu_bwd_kernel<<<grid1((long long)B * net->hidden), 256, 0, st>>>(net->t1, net->amlp,
                                                                       (long long)B * net->hidden, net->t2);
    // first dense layer
    NCK(net, (gemm<float, float, float, true, false>(st, net->hidden, net->flat, B, 1.f, net->t2, net->hidden,
                                                    net->h3, net->flat, 0.f, G + net->off[6], net->flat)));
    colsum_kernel<<<(net->hidden + 127) / 128, 128, 0, st>>>(net->t2, B, net->hidden, G + net->off[7]);
    NCK(net, (gemm<float, float, float, false, false>(st, B, net->flat, net->hidden, 1.f, net->t2, net->hidden,
                                                     P + net->off[6], net->flat, 0.f, net->t1, net->flat)));
    // convolutions, last to first: t1 holds dh of the layer's output
    const float* as[3] = {net->a1, net->a2, net->a3};
    const float* ins[3] = {net->x, net->h1, net->h2};
    for (int l = 2; l >= 0; --l) {
        const int cin = l == 0 ? 1 : net->c[l - 1], m = net->m[l + 1], nin = net->m[l];
        const long long cells = (long long)B * net->c[l] * m * m * m;
        relu_bwd_kernel<<<grid1(cells), 256, 0, st>>>(net->t1, as[l], cells, net->t2);   // da
        conv_bwd_w_kernel<<<net->c[l] * (cin * 27 + 1), 256, 0, st>>>(net->t2, ins[l], B, cin, nin,
                                                                       net->c[l], m, G + net->off[2 * l],
                                                                       G + net->off[2 * l + 1]);
        if (l > 0) {
            const long long icells = (long long)B * cin * nin * nin * nin;
            conv_bwd_data_kernel<<<grid1(icells), 256, 0, st>>>(net->t2, P + net->off[2 * l], B, cin, nin,
                                                                net->c[l], m, net->t1);
        }
    }
    NCK(net, cudaGetLastError());
    float h_loss = 0.f;
    NCK(net, cudaMemcpyAsync(&h_loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    if (grad_host)
        NCK(net, cudaMemcpyAsync(grad_host, G, net->off[10] * sizeof(float), cudaMemcpyDeviceToHost, st));
    NCK(net, cudaStreamSynchronize(st));
    if (loss) *loss = h_loss;
    return SFM_OK;
}

extern "C" int sfm_net_adam(sfm_net* net, float lr) {
    if (!net || !(lr > 0.f)) return nfail(net, SFM_ERR_ARG, "sfm_net_adam: bad arguments");
    NCK(net, cudaSetDevice(net->device));
    net->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->t), c2 = 1.f - powf(b2, (float)net->t);
    adam_kernel<<<grid1(net->off[10]), 256, 0, net->stream>>>(net->params, net->grads, net->am, net->av,
                                                              net->off[10], lr, b1, b2, 1e-8f, c1, c2);
    NCK(net, cudaGetLastError());
    net->pb_valid = false;
    return SFM_OK;
}

// Codes of a batch: z [B][code] (device).  bf16: BF16 weights and
// convolution activations with FP32 accumulation; else the FP32 pass.
extern "C" int sfm_net_forward(sfm_net* net, const float* c, int B, float* z, int bf16) {
    if (!net || !c || !z || B < 1) return nfail(net, SFM_ERR_ARG, "sfm_net_forward: bad arguments");
    NCK(net, cudaSetDevice(net->device));
    int rc = ensure_acts(net, B);
    if (rc) return rc;
    cudaStream_t st = net->stream;
    if (!bf16) {
        rc = forward_f32(net, c, B);
        if (rc) return rc;
    } else {
        if (!net->pb_valid) {
            to_bf16_kernel<<<grid1(net->off[10]), 256, 0, st>>>(net->params, net->pb, net->off[10]);
            net->pb_valid = true;
        }
        const __nv_bfloat16* P = net->pb;
        const long long n3 = (long long)net->n * net->n * net->n;
        features_kernel<__nv_bfloat16><<<grid1(B * n3), 256, 0, st>>>(c, 2500.f, B * n3, net->xb);
        const __nv_bfloat16* in = net->xb;
        __nv_bfloat16* hs[3] = {net->h1b, net->h2b, net->h3b};
        int cin = 1;
        for (int l = 0; l < 3; ++l) {
            const long long cells = (long long)B * net->c[l] * net->m[l + 1] * net->m[l + 1] * net->m[l + 1];
            conv_fwd_kernel<__nv_bfloat16, __nv_bfloat16><<<grid1(cells), 256, 0, st>>>(
                in, P + net->off[2 * l], P + net->off[2 * l + 1], B, cin, net->m[l], net->c[l],
                net->m[l + 1], nullptr, hs[l]);
            in = hs[l];
            cin = net->c[l];
        }
        NCK(net, cudaGetLastError());
        NCK(net, (gemm<float, __nv_bfloat16, __nv_bfloat16, false, true>(
                     st, B, net->hidden, net->flat, 1.f, net->h3b, net->flat, P + net->off[6], net->flat, 0.f,
                     net->hmlp, net->hidden, P + net->off[7], 1, nullptr)));
        NCK(net, (gemm<float, float, __nv_bfloat16, false, true>(st, B, net->code, net->hidden, 1.f, net->hmlp,
                                                                net->hidden, P + net->off[8], net->hidden, 0.f,
                                                                net->z, net->code, P + net->off[9], 0, nullptr)));
    }
    NCK(net, cudaMemcpyAsync(z, net->z, (size_t)B * net->code * sizeof(float), cudaMemcpyDeviceToDevice, st));
    NCK(net, cudaStreamSynchronize(st));
    return SFM_OK;
}

// ---------------------------------------------------------------------------
// Decoder targets, decoder fit and decoding (FP64)
// ---------------------------------------------------------------------------
namespace sfm {
namespace sur {

constexpr int SLD = 65;   // shared-memory row stride of a b x b block (b <= 64)

// raw numbers of block i of a set: blocks Gamma_2..Gamma_k then
// Gammahat_2..Gammahat_k (0-based levels 1..k-1); per block the strictly
// lower entries of U row by row, then log of the pivots, L = chol(B) = U D.
// A pivot at or below 1e-14 of the largest diagonal entry (a level that is
// semi-definite to rounding) is floored there.
__global__ void encode_kernel(const double* coef, int b, int k, double* raw) {
    __shared__ double A[64 * SLD];
    __shared__ double s_max;
    const int set = blockIdx.y, i = blockIdx.x;
    const int lev = 1 + (i % (k - 1)), kind = i / (k - 1);
    const double* B = coef + (long long)set * 2 * k * b * b + ((long long)kind * k + lev) * b * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e / b, c = e % b;
        A[r * SLD + c] = 0.5 * (B[r * b + c] + B[c * b + r]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int r = 0; r < b; ++r) mx = fmax(mx, A[r * SLD + r]);
        s_max = mx;
    }
    __syncthreads();
    const double floor_ = 1e-14 * s_max;
    for (int c = 0; c < b; ++c) {
        double d = A[c * SLD + c];
        __syncthreads();
        if (!(d > floor_)) d = floor_;
        const double l = sqrt(d);
        if (threadIdx.x == 0) A[c * SLD + c] = l;
        for (int r = c + 1 + threadIdx.x; r < b; r += blockDim.x) A[r * SLD + c] /= l;
        __syncthreads();
        const int rest = b - c - 1;
        for (int t = threadIdx.x; t < rest * rest; t += blockDim.x) {
            const int r = c + 1 + t / rest, cc = c + 1 + t % rest;
            if (cc <= r) A[r * SLD + cc] -= A[r * SLD + c] * A[cc * SLD + c];
        }
        __syncthreads();
    }
    const long long nlow = (long long)b * (b - 1) / 2, nper = nlow + b;
    double* out = raw + (long long)set * 2 * (k - 1) * nper + (long long)i * nper;
    for (int e = threadIdx.x; e < nlow; e += blockDim.x) {
        // row r >= 1 holds entries (r, 0..r-1) starting at r(r-1)/2
        int r = (int)((1.0 + sqrt(1.0 + 8.0 * e)) * 0.5);
        while ((long long)r * (r - 1) / 2 > e) --r;
        while ((long long)(r + 1) * r / 2 <= e) ++r;
        const int c = (int)(e - (long long)r * (r - 1) / 2);
        out[e] = A[r * SLD + c] / A[c * SLD + c];
    }
    for (int r = threadIdx.x; r < b; r += blockDim.x) out[nlow + r] = log(A[r * SLD + r]);
}

// block i of set `set` from its raw numbers: L = U diag(exp(g)), B = L L^T,
// written at its level in the coefficient layout
__global__ void decode_blocks_kernel(const double* raw, int b, int k, double* coef) {
    __shared__ double L[64 * SLD];
    const int set = blockIdx.y, i = blockIdx.x;
    const int lev = 1 + (i % (k - 1)), kind = i / (k - 1);
    const long long nlow = (long long)b * (b - 1) / 2, nper = nlow + b;
    const double* v = raw + (long long)set * 2 * (k - 1) * nper + (long long)i * nper;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e / b, c = e % b;
        double u = r == c ? 1.0 : (c < r ? v[(long long)r * (r - 1) / 2 + c] : 0.0);
        L[r * SLD + c] = u * exp(v[nlow + c]);
    }
    __syncthreads();
    double* B = coef + (long long)set * 2 * k * b * b + ((long long)kind * k + lev) * b * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e / b, c = e % b;
        double s = 0.0;
        const int top = r < c ? r : c;
        for (int t = 0; t <= top; ++t) s += L[r * SLD + t] * L[c * SLD + t];
        B[e] = s;
    }
}

// column means of X [N][n]
__global__ void colmean_kernel(const double* X, long long N, long long n, double* mu) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long r = 0; r < N; ++r) s += X[r * n + c];
        mu[c] = s / (double)N;
    }
}

// Y[r][c] = X[r][c] - mu[c] (sign -1) or + mu[c] (sign +1)
__global__ void shift_rows_kernel(const double* X, const double* mu, long long N, long long n, double sign,
                                  double* Y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N * n;
         i += (long long)gridDim.x * blockDim.x)
        Y[i] = X[i] + sign * mu[i % n];
}

// seeded standard normal numbers (a counter-based hash and Box-Muller)
__global__ void gauss_kernel(double* out, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        auto h = [](unsigned long long z) {
            z += 0x9e3779b97f4a7c15ull;
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
            return z ^ (z >> 31);
        };
        const unsigned long long a = h(seed * 0x100000001b3ull + 2 * (unsigned long long)i);
        const unsigned long long b2 = h(seed * 0x100000001b3ull + 2 * (unsigned long long)i + 1);
        const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((b2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        out[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
}

// upper Cholesky factor R of the d x d Gram matrix G (G = R^T R), one block;
// *bad set when a pivot is not positive
__global__ void gram_chol_kernel(double* G, int d, int* bad) {
    for (int c = 0; c < d; ++c) {
        __syncthreads();
        const double dd = G[c * d + c];
        __syncthreads();
        if (!(dd > 0.0)) {
            if (threadIdx.x == 0) *bad = 1;
            return;
        }
        const double l = sqrt(dd);
        __syncthreads();
        if (threadIdx.x == 0) G[c * d + c] = l;
        for (int j = c + 1 + threadIdx.x; j < d; j += blockDim.x) G[c * d + j] /= l;
        __syncthreads();
        for (int t = threadIdx.x; t < (d - c - 1) * (d - c - 1); t += blockDim.x) {
            const int i = c + 1 + t / (d - c - 1), j = c + 1 + t % (d - c - 1);
            if (j >= i) G[i * d + j] -= G[c * d + i] * G[c * d + j];
        }
    }
}

// Q[r][:] <- Q[r][:] R^{-1} (R upper triangular d x d): forward substitution
// per row
__global__ void rsolve_kernel(double* Q, long long rows, int d, const double* R) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        double* q = Q + r * d;
        for (int j = 0; j < d; ++j) {
            double s = q[j];
            for (int t = 0; t < j; ++t) s -= q[t] * R[t * d + j];
            q[j] = s / R[j * d + j];
        }
    }
}

// per-column RMS of the (centred) codes C [N][d]; zero columns give 1
__global__ void code_rms_kernel(const double* C, int N, int d, double* sd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    for (int r = 0; r < N; ++r) s += C[(long long)r * d + c] * C[(long long)r * d + c];
    s = sqrt(s / N);
    sd[c] = s > 0.0 ? s : 1.0;
}

// P[r][c] *= sd[c] (rows = nraw) and C[r][c] /= sd[c] (rows = N)
__global__ void rescale_kernel(double* P, long long nraw, double* C, int N, int d, const double* sd) {
    const long long total = nraw * d + (long long)N * d;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < nraw * d) P[i] *= sd[i % d];
        else {
            const long long j = i - nraw * d;
            C[j] /= sd[j % d];
        }
    }
}

__global__ void f64_to_f32_kernel(const double* in, float* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void f32_to_f64_kernel(const float* in, double* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

}  // namespace sur
}  // namespace sfm

// ---------------------------------------------------------------------------
// NtD map of an S-fraction at complex lambda (Eq. 15's transfer function by
// the continued fraction in the file comment), one block per (set, lambda)
// ---------------------------------------------------------------------------
namespace sfm {
namespace sur {

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    const double d = cabs2(b);
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// In-place inverse of the b x b complex matrix A (row stride b) by
// Gauss-Jordan elimination with partial (row) pivoting; the row swaps are
// undone on the columns at the end.  All threads of the block take part.
__device__ void cinv(cplx* A, int b, int* perm) {
    __shared__ int s_p;
    for (int c = 0; c < b; ++c) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int p = c;
            double best = cabs2(A[c * b + c]);
            for (int r = c + 1; r < b; ++r) {
                const double v = cabs2(A[r * b + c]);
                if (v > best) { best = v; p = r; }
            }
            s_p = p;
            perm[c] = p;
        }
        __syncthreads();
        const int p = s_p;
        if (p != c)
            for (int j = threadIdx.x; j < b; j += blockDim.x) {
                const cplx t = A[c * b + j];
                A[c * b + j] = A[p * b + j];
                A[p * b + j] = t;
            }
        __syncthreads();
        const cplx piv = A[c * b + c];
        __syncthreads();
        if (threadIdx.x == 0) A[c * b + c] = {1.0, 0.0};
        __syncthreads();
        for (int j = threadIdx.x; j < b; j += blockDim.x) A[c * b + j] = cdiv(A[c * b + j], piv);
        __syncthreads();
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
            const int r = t / b, j = t % b;
            if (r == c || j == c) continue;
            A[r * b + j] = csub(A[r * b + j], cmul(A[r * b + c], A[c * b + j]));
        }
        __syncthreads();
        for (int r = threadIdx.x; r < b; r += blockDim.x)
            if (r != c) {
                const cplx f = A[r * b + c];
                A[r * b + c] = cmul({-f.re, -f.im}, A[c * b + c]);
            }
    }
    __syncthreads();
    for (int c = b - 1; c >= 0; --c) {
        const int p = perm[c];
        if (p != c)
            for (int r = threadIdx.x; r < b; r += blockDim.x) {
                const cplx t = A[r * b + c];
                A[r * b + c] = A[r * b + p];
                A[r * b + p] = t;
            }
        __syncthreads();
    }
}

// S(lambda) of set `set` for lambda index `li` into S [set][lam][b][b]
__global__ void sfrac_transfer_kernel(const double* coef, int b, int k, const double* lam, int nlam,
                                      double* S) {
    extern __shared__ __align__(16) unsigned char ntd_smem[];
    cplx* Y = reinterpret_cast<cplx*>(ntd_smem);
    cplx* W = Y + b * b;
    __shared__ int perm[64];
    const int set = blockIdx.y, li = blockIdx.x;
    const cplx L = {lam[2 * li], lam[2 * li + 1]};
    const double* G = coef + (long long)set * 2 * k * b * b;      // Gamma_j at G + j b^2
    const double* Gh = G + (long long)k * b * b;                  // Gammahat_j
    const int bb = b * b;
    // Y = lambda Gammahat_k^{-1} + Gamma_k
    for (int e = threadIdx.x; e < bb; e += blockDim.x) W[e] = {Gh[(long long)(k - 1) * bb + e], 0.0};
    cinv(W, b, perm);
    __syncthreads();
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const cplx t = cmul(L, W[e]);
        Y[e] = {t.re + G[(long long)(k - 1) * bb + e], t.im};
    }
    for (int j = k - 2; j >= 0; --j) {
        __syncthreads();
        for (int e = threadIdx.x; e < bb; e += blockDim.x) W[e] = Y[e];
        cinv(W, b, perm);                                  // W = Y_{j+1}^{-1}
        __syncthreads();
        for (int e = threadIdx.x; e < bb; e += blockDim.x) Y[e] = {G[(long long)j * bb + e], 0.0};
        cinv(Y, b, perm);                                  // Y = Gamma_j^{-1}
        __syncthreads();
        for (int e = threadIdx.x; e < bb; e += blockDim.x) W[e] = {W[e].re + Y[e].re, W[e].im + Y[e].im};
        cinv(W, b, perm);                                  // W = (Gamma_j^{-1} + Y_{j+1}^{-1})^{-1}
        __syncthreads();
        for (int e = threadIdx.x; e < bb; e += blockDim.x) Y[e] = {Gh[(long long)j * bb + e], 0.0};
        cinv(Y, b, perm);                                  // Y = Gammahat_j^{-1}
        __syncthreads();
        for (int e = threadIdx.x; e < bb; e += blockDim.x) {
            const cplx t = cmul(L, Y[e]);
            Y[e] = {t.re + W[e].re, t.im + W[e].im};
        }
    }
    __syncthreads();
    cinv(Y, b, perm);                                      // S = Y_1^{-1}
    __syncthreads();
    double* out = S + ((long long)set * nlam + li) * 2 * bb;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        out[2 * e] = Y[e].re;
        out[2 * e + 1] = Y[e].im;
    }
}

// err[i] = |A_i - R_i|_F / |R_i|_F over complex b x b matrices
__global__ void rel_frob_kernel(const double* A, const double* R, int bb2, int count, double* err) {
    __shared__ double na[256], nr[256];
    const int i = blockIdx.x;
    double a = 0.0, r = 0.0;
    for (int e = threadIdx.x; e < bb2; e += blockDim.x) {
        const double d = A[(long long)i * bb2 + e] - R[(long long)i * bb2 + e];
        a += d * d;
        r += R[(long long)i * bb2 + e] * R[(long long)i * bb2 + e];
    }
    na[threadIdx.x] = a;
    nr[threadIdx.x] = r;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { na[threadIdx.x] += na[threadIdx.x + s]; nr[threadIdx.x] += nr[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) err[i] = sqrt(na[0] / nr[0]);
}

cudaError_t launch_transfer(const double* coef, int count, int b, int k, const double* d_lam, int nlam,
                            double* S, cudaStream_t st) {
    const size_t smem = 2 * (size_t)b * b * sizeof(cplx);
    cudaError_t e = cudaFuncSetAttribute(sfrac_transfer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    for (int s0 = 0; s0 < count; s0 += 65535) {
        const int ns = std::min(65535, count - s0);
        sfrac_transfer_kernel<<<dim3(nlam, ns), 256, smem, st>>>(coef + (long long)s0 * 2 * k * b * b, b, k,
                                                                 d_lam, nlam,
                                                                 S + (long long)s0 * nlam * 2 * b * b);
    }
    return cudaGetLastError();
}

}  // namespace sur
}  // namespace sfm

namespace {
int gfail(int code, const std::string& msg) {
    sfm::set_global_error(msg);
    return code;
}
#define GCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e__ = (call);                                                                \
        if (e__ != cudaSuccess)                                                                  \
            return gfail(e__ == cudaErrorMemoryAllocation ? SFM_ERR_NOMEM : SFM_ERR_CUDA,        \
                         std::string(#call) + ": " + cudaGetErrorString(e__));                   \
    } while (0)

long long raw_size(int b, int k) { return 2LL * (k - 1) * ((long long)b * (b - 1) / 2 + b); }
}  // namespace

extern "C" int sfm_raw_encode(int device, int count, int b, int k, const double* coef, double* raw) {
    if (count < 1 || b < 1 || b > 64 || k < 2 || !coef || !raw)
        return gfail(SFM_ERR_ARG, "sfm_raw_encode: bad arguments");
    GCK(cudaSetDevice(device));
    for (int s0 = 0; s0 < count; s0 += 65535) {
        const int ns = std::min(65535, count - s0);
        sfm::sur::encode_kernel<<<dim3(2 * (k - 1), ns), 256>>>(coef + (long long)s0 * 2 * k * b * b, b, k,
                                                                raw + (long long)s0 * raw_size(b, k));
    }
    GCK(cudaGetLastError());
    GCK(cudaDeviceSynchronize());
    return SFM_OK;
}

extern "C" int sfm_net_fit_decoder(sfm_net* net, int b, int k, const double* raw, int N, int iters,
                                   unsigned long long seed, float* codes) {
    if (!net || b < 1 || b > 64 || k < 2 || !raw || N < net->code || iters < 0)
        return nfail(net, SFM_ERR_ARG, "sfm_net_fit_decoder: bad arguments (N >= code needed)");
    NCK(net, cudaSetDevice(net->device));
    cudaStream_t st = net->stream;
    const long long nraw = raw_size(b, k);
    const int d = net->code;
    net->b = b;
    net->k = k;
    net->nraw = (int)nraw;
    double *Rc = nullptr, *Z = nullptr, *G = nullptr, *C64 = nullptr;
    int* bad = nullptr;
    auto cleanup = [&]() { nfree(Rc); nfree(Z); nfree(G); nfree(C64); nfree(bad); };
#define FCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e__ = (call);                                                                \
        if (e__ != cudaSuccess) {                                                                \
            cleanup();                                                                           \
            return nfail(net, SFM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
        }                                                                                        \
    } while (0)
    FCK(nalloc(net->mu, nraw));
    FCK(nalloc(net->P, nraw * d));
    FCK(nalloc(Rc, (long long)N * nraw));
    FCK(nalloc(Z, (long long)N * d));
    FCK(nalloc(G, (long long)d * d));
    FCK(nalloc(C64, (long long)N * d));
    FCK(nalloc(bad, 1));
    FCK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    colmean_kernel<<<grid1(nraw), 256, 0, st>>>(raw, N, nraw, net->mu);
    shift_rows_kernel<<<grid1((long long)N * nraw), 256, 0, st>>>(raw, net->mu, N, nraw, -1.0, Rc);
    // randomized subspace iteration for the range of Rc^T: Q = Rc^T Omega,
    // then Q <- orth(Rc^T (Rc Q)), orthonormalised by Cholesky QR twice
    gauss_kernel<<<grid1((long long)N * d), 256, 0, st>>>(Z, (long long)N * d, seed);
    FCK((dgemm<true, false>(st, (int)nraw, d, N, 1.0, Rc, (int)nraw, Z, d, 0.0, net->P, d)));
    auto orth = [&]() -> cudaError_t {
        for (int pass = 0; pass < 2; ++pass) {
            cudaError_t e = dgemm<true, false>(st, d, d, (int)nraw, 1.0, net->P, d, net->P, d, 0.0, G, d);
            if (e != cudaSuccess) return e;
            gram_chol_kernel<<<1, 256, 0, st>>>(G, d, bad);
            rsolve_kernel<<<grid1(nraw), 256, 0, st>>>(net->P, nraw, d, G);
        }
        return cudaGetLastError();
    };
    FCK(orth());
    for (int it = 0; it < iters; ++it) {
        FCK((dgemm<false, false>(st, N, d, (int)nraw, 1.0, Rc, (int)nraw, net->P, d, 0.0, Z, d)));
        FCK((dgemm<true, false>(st, (int)nraw, d, N, 1.0, Rc, (int)nraw, Z, d, 0.0, net->P, d)));
        FCK(orth());
    }
    int hbad = 0;
    FCK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    if (hbad) {
        cleanup();
        return nfail(net, SFM_ERR_BREAKDOWN, "sfm_net_fit_decoder: rank-deficient targets");
    }
    // codes of the targets, then each code coordinate scaled to unit RMS
    // over the targets (P's column scaled back, so mu + P z is unchanged):
    // the network then learns numbers of order one
    FCK((dgemm<false, false>(st, N, d, (int)nraw, 1.0, Rc, (int)nraw, net->P, d, 0.0, C64, d)));
    code_rms_kernel<<<(d + 127) / 128, 128, 0, st>>>(C64, N, d, G);
    rescale_kernel<<<grid1(nraw * d + (long long)N * d), 256, 0, st>>>(net->P, nraw, C64, N, d, G);
    FCK(cudaGetLastError());
    if (codes) {
        f64_to_f32_kernel<<<grid1((long long)N * d), 256, 0, st>>>(C64, codes, (long long)N * d);
        FCK(cudaGetLastError());
    }
    FCK(cudaStreamSynchronize(st));
#undef FCK
    cleanup();
    return SFM_OK;
}

extern "C" int sfm_net_decode(sfm_net* net, const float* z, int B, double* coef) {
    if (!net || !z || B < 1 || !coef) return nfail(net, SFM_ERR_ARG, "sfm_net_decode: bad arguments");
    if (!net->P) return nfail(net, SFM_ERR_STATE, "sfm_net_decode: no decoder fitted");
    NCK(net, cudaSetDevice(net->device));
    cudaStream_t st = net->stream;
    const int d = net->code;
    const long long nraw = net->nraw;
    double *z64 = nullptr, *R = nullptr;
    NCK(net, nalloc(z64, (long long)B * d));
    cudaError_t e = nalloc(R, (long long)B * nraw);
    if (e == cudaSuccess) {
        f32_to_f64_kernel<<<grid1((long long)B * d), 256, 0, st>>>(z, z64, (long long)B * d);
        // raw = mu + P z for every sample
        e = dgemm<false, true>(st, B, (int)nraw, d, 1.0, z64, d, net->P, d, 0.0, R, (int)nraw);
    }
    if (e == cudaSuccess) {
        shift_rows_kernel<<<grid1((long long)B * nraw), 256, 0, st>>>(R, net->mu, B, nraw, 1.0, R);
        for (int s0 = 0; s0 < B; s0 += 65535) {
            const int ns = std::min(65535, B - s0);
            decode_blocks_kernel<<<dim3(2 * (net->k - 1), ns), 256, 0, st>>>(
                R + (long long)s0 * nraw, net->b, net->k, coef + (long long)s0 * 2 * net->k * net->b * net->b);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    nfree(z64);
    nfree(R);
    if (e != cudaSuccess) return nfail(net, SFM_ERR_CUDA, std::string("sfm_net_decode: ") + cudaGetErrorString(e));
    return SFM_OK;
}

extern "C" int sfm_ntd_error(int device, int count, int b, int k, const double* coef_a,
                             const double* coef_r, int nlam, const double* lam, double* err) {
    if (count < 1 || b < 1 || b > 64 || k < 1 || !coef_a || !coef_r || nlam < 1 || !lam || !err)
        return gfail(SFM_ERR_ARG, "sfm_ntd_error: bad arguments");
    GCK(cudaSetDevice(device));
    const long long per = 2LL * b * b;
    double *d_lam = nullptr, *Sa = nullptr, *Sr = nullptr, *d_err = nullptr;
    auto cleanup = [&]() { nfree(d_lam); nfree(Sa); nfree(Sr); nfree(d_err); };
    cudaError_t e = nalloc(d_lam, 2 * (size_t)nlam);
    if (e == cudaSuccess) e = nalloc(Sa, (size_t)count * nlam * per);
    if (e == cudaSuccess) e = nalloc(Sr, (size_t)count * nlam * per);
    if (e == cudaSuccess) e = nalloc(d_err, (size_t)count * nlam);
    if (e == cudaSuccess) e = cudaMemcpy(d_lam, lam, 2 * nlam * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = sfm::sur::launch_transfer(coef_a, count, b, k, d_lam, nlam, Sa, 0);
    if (e == cudaSuccess) e = sfm::sur::launch_transfer(coef_r, count, b, k, d_lam, nlam, Sr, 0);
    if (e == cudaSuccess) {
        sfm::sur::rel_frob_kernel<<<count * nlam, 256>>>(Sa, Sr, (int)per, count * nlam, d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(err, d_err, (size_t)count * nlam * sizeof(double), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return gfail(SFM_ERR_CUDA, std::string("sfm_ntd_error: ") + cudaGetErrorString(e));
    return SFM_OK;
}

// ---------------------------------------------------------------------------
// helpers for the builder's surrogate mode
// ---------------------------------------------------------------------------
namespace sfm {
namespace sur {

// err[i] = |S_i(sigma) - Sref_i|_F / |Sref_i|_F, S_i the transfer function of
// coefficient set i (complex evaluation at lambda = sigma, imaginary part 0)
// and Sref_i a real b x b matrix
// err[i] = max(|S_i(sigma) - Sref_i| / |Sref_i|, |S_i'(sigma) - Dref_i| / |Dref_i|)
// (Frobenius norms): S_i the transfer function of coefficient set i, its
// derivative by the central difference of the values at sigma (1 -+ eps)
// (S holds nl = 1 or 3 lambdas per set, complex with zero imaginary part),
// Sref, Dref real b x b (Dref NULL: the value alone)
__global__ void sigma_err_kernel(const double* S, const double* Sref, int bb, int nl, const double* Dref,
                                 double dl, double* err) {
    __shared__ double na[256], nr[256], ma[256], mr[256];
    const int i = blockIdx.x;
    const double* s0 = S + (long long)i * nl * 2 * bb;
    double a = 0.0, r = 0.0, c = 0.0, q = 0.0;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const double re = s0[2 * e], im = s0[2 * e + 1];
        const double f = Sref[(long long)i * bb + e];
        a += (re - f) * (re - f) + im * im;
        r += f * f;
        if (Dref) {
            const double dv = (s0[4 * bb + 2 * e] - s0[2 * bb + 2 * e]) / dl;
            const double g = Dref[(long long)i * bb + e];
            c += (dv - g) * (dv - g);
            q += g * g;
        }
    }
    na[threadIdx.x] = a;
    nr[threadIdx.x] = r;
    ma[threadIdx.x] = c;
    mr[threadIdx.x] = q;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            na[threadIdx.x] += na[threadIdx.x + s];
            nr[threadIdx.x] += nr[threadIdx.x + s];
            ma[threadIdx.x] += ma[threadIdx.x + s];
            mr[threadIdx.x] += mr[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = sqrt(na[0] / nr[0]);
        if (Dref) v = fmax(v, sqrt(ma[0] / mr[0]));
        err[i] = v;
    }
}

}  // namespace sur

int net_shape(const sfm_net* net, int* n, int* b, int* k) {
    if (!net || !net->P) return SFM_ERR_STATE;
    *n = net->n;
    *b = net->b;
    *k = net->k;
    return SFM_OK;
}

int net_code_dim(const sfm_net* net) { return net ? net->code : 0; }

cudaError_t sigma_check(const double* sets, int count, int b, int k, double sigma, const double* Sref,
                        const double* Dref, double* err, cudaStream_t st) {
    // lambda = sigma, and sigma (1 -+ eps) for the central difference of S
    const double eps = 1e-4;
    const int nl = Dref ? 3 : 1;
    double *lam = nullptr, *S = nullptr;
    cudaError_t e = nalloc(lam, 6);
    if (e == cudaSuccess) e = nalloc(S, (size_t)count * nl * 2 * b * b);
    const double hl[6] = {sigma, 0.0, sigma * (1.0 - eps), 0.0, sigma * (1.0 + eps), 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam, hl, sizeof(hl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = sur::launch_transfer(sets, count, b, k, lam, nl, S, st);
    if (e == cudaSuccess) {
        sur::sigma_err_kernel<<<count, 256, 0, st>>>(S, Sref, b * b, nl, Dref, 2.0 * sigma * eps, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    nfree(lam);
    nfree(S);
    return e;
}

}  // namespace sfm
