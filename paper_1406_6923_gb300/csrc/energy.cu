// Discrete energy of the coupled leapfrog (the conserved quantity of Stage 2,
// written for the assembled system of Eqs. 17-19):
//   E^{n+1/2} = 1/2 (delta/dt)^T MM (delta/dt) + 1/2 (U^{n+1})^T KK U^n,
// delta = U^{n+1} - U^n.  Both forms are sums over subdomains:
//   KK = sum_s E_s^T D^T Gamma D E_s, so U^T KK V = sum_s sum_j
//        Delta_j(U)^T Gamma_j Delta_j(V), Delta_j = U_{j+1} - U_j (U_{k+1} = 0);
//   MM = blockdiag(Gammahat_j^{-1} (j >= 2), H_f^{-1} (shared faces),
//        [Gammahat_1]_f^{-1} (outer faces)), and H_f^{-1} is the sum of both
//        sides' [Gammahat_1]_f^{-1}, so with each side holding its own copy of
//        the face blocks delta^T MM delta = sum_s sum_j delta_j^T
//        Gammahat_j^{-1} delta_j (Gammahat_1 is block diagonal over faces).
// One block per (shot, subdomain, level) evaluates its two terms in FP64
// (Cholesky of Gammahat_j, forward substitution); the host adds them in a
// fixed order.
#include "sfm_internal.h"

namespace sfm {

constexpr int EN_LD = 65;

__global__ void __launch_bounds__(64) energy_terms_kernel(const double* coef, const long long* coef_off,
                                                          const int* sub_b, const int* sub_k, int nsub,
                                                          int kmax, const double* U, const double* D,
                                                          long long stride, const long long* state_off,
                                                          int u_base, double* out) {
    __shared__ double A[64 * EN_LD];
    __shared__ double x[64], y[64], red[64];
    __shared__ int s_ok;
    const int j = blockIdx.x, u = u_base + (int)blockIdx.y;
    const int q = u / nsub, s = u - q * nsub;
    const int b = sub_b[s], k = sub_k[s];
    double* o = out + ((long long)u * kmax + j) * 2;
    if (j >= k) {
        if (threadIdx.x == 0) { o[0] = 0.0; o[1] = 0.0; }
        return;
    }
    const double* un = U + q * stride + state_off[s];     // U^{n+1}
    const double* dl = D + q * stride + state_off[s];     // delta = U^{n+1} - U^n
    const int i = threadIdx.x;
    // potential term: Delta_j(U^{n+1})^T Gamma_j Delta_j(U^n)
    if (i < b) {
        const double a1 = (j + 1 < k) ? un[(j + 1) * b + i] : 0.0;
        const double d1 = (j + 1 < k) ? dl[(j + 1) * b + i] : 0.0;
        const double a0 = un[j * b + i], d0 = dl[j * b + i];
        x[i] = (a1 - d1) - (a0 - d0);          // Delta_j(U^n)
        y[i] = a1 - a0;                        // Delta_j(U^{n+1})
    }
    __syncthreads();
    const double* G = coef + coef_off[s] + (long long)j * b * b;
    double pot = 0.0;
    if (i < b) {
        double r = 0.0;
        for (int c = 0; c < b; ++c) r += G[i * b + c] * x[c];
        pot = y[i] * r;
    }
    red[i] = pot;
    __syncthreads();
    if (i == 0) {
        double t = 0.0;
        for (int c = 0; c < 64; ++c) t += red[c];
        o[1] = t;
    }
    // kinetic term: delta_j^T Gammahat_j^{-1} delta_j = |L^{-1} delta_j|^2
    const double* Gh = coef + coef_off[s] + (long long)(k + j) * b * b;
    for (int e = i; e < b * b; e += 64) A[(e / b) * EN_LD + e % b] = Gh[e];
    if (i == 0) s_ok = 1;
    __syncthreads();
    for (int c = 0; c < b; ++c) {
        const double d = A[c * EN_LD + c];
        __syncthreads();
        if (!(d > 0.0)) {
            if (i == 0) s_ok = 0;
            break;
        }
        const double l = sqrt(d);
        if (i == 0) A[c * EN_LD + c] = l;
        for (int r = c + 1 + i; r < b; r += 64) A[r * EN_LD + c] /= l;
        __syncthreads();
        for (int t = i; t < (b - c - 1) * (b - c - 1); t += 64) {
            const int r = c + 1 + t / (b - c - 1), cc = c + 1 + t % (b - c - 1);
            if (cc <= r) A[r * EN_LD + cc] -= A[r * EN_LD + c] * A[cc * EN_LD + c];
        }
        __syncthreads();
    }
    __syncthreads();
    if (i == 0) {
        if (!s_ok) {
            o[0] = nan("");
        } else {
            double t = 0.0;
            for (int r = 0; r < b; ++r) {
                double v = dl[j * b + r];
                for (int c = 0; c < r; ++c) v -= A[r * EN_LD + c] * y[c];
                v /= A[r * EN_LD + r];
                y[r] = v;
                t += v * v;
            }
            o[0] = t;
        }
    }
}

cudaError_t launch_energy_terms(const double* coef, const long long* coef_off, const int* sub_b,
                                const int* sub_k, int nsub, int kmax, int nshots, const double* U,
                                const double* D, long long stride, const long long* state_off,
                                double* out, cudaStream_t st) {
    const int units = nshots * nsub;
    for (int u0 = 0; u0 < units; u0 += 65535) {
        const int nu = units - u0 < 65535 ? units - u0 : 65535;
        energy_terms_kernel<<<dim3(kmax, nu), 64, 0, st>>>(coef, coef_off, sub_b, sub_k, nsub, kmax, U,
                                                           D, stride, state_off, u0, out);
    }
    return cudaGetLastError();
}

template <typename T>
__device__ __forceinline__ double as_f64(T v) { return (double)v; }
template <>
__device__ __forceinline__ double as_f64<float2>(float2 v) { return (double)v.x + (double)v.y; }

template <typename T>
__global__ void state_to_f64_kernel(const T* in, double* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = as_f64(in[i]);
}

template <typename T>
cudaError_t launch_state_to_f64(const T* in, double* out, size_t n, cudaStream_t st) {
    int grid = (int)((n + 255) / 256);
    if (grid > 8192) grid = 8192;
    if (grid < 1) grid = 1;
    state_to_f64_kernel<T><<<grid, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template cudaError_t launch_state_to_f64<float>(const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_state_to_f64<float2>(const float2*, double*, size_t, cudaStream_t);

}  // namespace sfm
