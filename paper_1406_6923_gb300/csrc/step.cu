// Coupled leapfrog stepping of all subdomain ROMs in matrix S-fraction form
// (Algorithm 1 stage 2; Eqs. 12, 18, 19).
//
// One persistent cooperative kernel runs all time steps.  Work units are
// (shot, subdomain) pairs spread over the blocks.  Per step n:
//
//   phase A (per unit, no cross-unit data):
//     Delta_j = U_{j+1} - U_j (U_{k+1} = 0),  phi_j = Gamma_j Delta_j      (Eq. 12)
//     mail    = phi_1 + p_1 f(t_n)            -- face data, step (2.1)
//     a_j     = Gammahat_j (phi_j - phi_{j-1} + p_j f(t_n)), j >= 2  (Eq. 19, step 2.2)
//     delta_j += dt^2 a_j,  U_j^{n+1} = U_j^n + delta_j
//   device-wide barrier (the exchange of step 2.1)
//   phase B (per unit, reads the neighbours' mail):
//     a_f = H_f (mail_f(self) + mail_f(neighbour))  (outer face: own term)  (Eq. 18)
//     delta_1,f += dt^2 a_f,  U_1,f^{n+1} = U_1,f^n + delta_1,f
//     plus this block's share of the receiver readout of U^n
//
// Each subdomain keeps its own copy of its level-1 face blocks; both sides
// of a shared face compute the same sum of the same two mail vectors with
// the same H_f copy, so the two copies stay bitwise equal (the continuity
// condition of Eq. 17).  U^n lives in buffer n % 3 and the mail in buffer
// n % 2: a block that runs ahead into phase A of step n+1 then never writes
// what a slower block still reads in phase B of step n, so one barrier per
// step suffices.
#include "sfm_internal.h"

#include <cooperative_groups.h>

namespace sfm {

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int* p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded device-wide barrier.  Returns false (and sets *err) when the
// barrier did not complete within timeout_ns, or when another block
// reported an error; every block then leaves the kernel.
__device__ bool grid_barrier(unsigned int* bar, unsigned int target, int* err,
                             unsigned long long timeout_ns, int skip_arrive) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if ((int)blockIdx.x != skip_arrive) red_release_add_u32(bar, 1u);
        int ok = 1;
        unsigned long long t0 = global_ns();
        while (ld_acquire_u32(bar) < target) {
            if (*(volatile int*)err != 0) { ok = 0; break; }
            if (global_ns() - t0 > timeout_ns) {
                atomicCAS(err, 0, (int)SFM_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    }
    return s;  // valid in thread 0
}

// Sum over the block in the policy's arithmetic (fixed order); valid in thread 0.
template <class P>
__device__ __forceinline__ typename P::C block_sum_p(typename P::C v, typename P::C* red) {
    for (int o = 16; o > 0; o >>= 1) v = P::add(v, P::shfl_xor(v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    typename P::C s = P::zero();
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = P::add(s, red[w]);
    }
    return s;
}

// Receiver readout of U (buffer `Ubuf`) at sample n for this block's share of
// (shot, pair) items.
template <class P>
__device__ void readout(const StepParams<typename P::S>& p, const typename P::S* Ubuf, int n,
                        typename P::C* red) {
    using C = typename P::C;
    const long long items = (long long)p.nshots * p.nrpairs;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int q = (int)(it / p.nrpairs), r = (int)(it % p.nrpairs);
        const int s = p.rp_sub[r];
        const int kb = p.sub_k[s] * p.sub_b[s];
        const typename P::S* row = p.rrows + p.rp_off[r];
        const typename P::S* U = Ubuf + q * p.state_stride + p.state_off[s];
        typename P::Acc acc = P::acc0();
        for (int t = threadIdx.x; t < kb; t += blockDim.x) P::fma(acc, P::ld(row + t), P::ld(U + t));
        const C v = block_sum_p<P>(P::get(acc), red);
        if (threadIdx.x == 0)
            P::st(p.partial + ((long long)q * (p.nsteps + 1) + n) * p.nrpairs + r, v);
    }
}

template <class P>
__global__ void __launch_bounds__(256) step_kernel(StepParams<typename P::S> p) {
    using S = typename P::S;
    using C = typename P::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sU = reinterpret_cast<C*>(smem_raw);              // (kmax+1)*bmax
    C* sD = sU + (p.kmax + 1) * p.bmax;                  // kmax*bmax: Delta, then psi
    C* sPhi = sD + p.kmax * p.bmax;                      // kmax*bmax
    C* red = sPhi + p.kmax * p.bmax;                     // 32
    const C dt2 = P::from_d(p.dt2);

    for (int n = 0; n < p.nsteps; ++n) {
        const S* Ucur = p.U[n % 3];
        S* Unxt = p.U[(n + 1) % 3];
        S* mail = (n & 1) ? p.mail1 : p.mail0;

        // ---------------- phase A ----------------
        for (int u = blockIdx.x; u < p.nunits; u += gridDim.x) {
            const int q = u / p.nsub, s = u - q * p.nsub;
            const int b = p.sub_b[s], k = p.sub_k[s], kb = k * b;
            const long long so = q * p.state_stride + p.state_off[s];
            const S* Uc = Ucur + so;
            S* Un = Unxt + so;
            S* dU = p.dU + so;
            const S* G = p.coef + p.coef_off[s];            // Gamma_j at G + j*b*b
            const S* Gh = G + (long long)k * b * b;          // Gammahat_j at Gh + j*b*b
            const long long sof = p.src_off[(long long)q * p.nsub + s];
            const C w = P::ld(p.wavelet + (long long)q * p.nsteps + n);
            __syncthreads();
            for (int t = threadIdx.x; t < kb; t += blockDim.x) sU[t] = P::ld(Uc + t);
            for (int t = threadIdx.x; t < b; t += blockDim.x) sU[kb + t] = P::zero();
            __syncthreads();
            for (int t = threadIdx.x; t < kb; t += blockDim.x) sD[t] = P::sub(sU[t + b], sU[t]);
            __syncthreads();
            // phi_j = Gamma_j Delta_j, j = 1..k  (Gamma symmetric: column-major = row-major)
            for (int t = threadIdx.x; t < kb; t += blockDim.x) {
                const int j = t / b, i = t - j * b;
                const S* Gj = G + (long long)j * b * b + i;
                const C* dj = sD + j * b;
                typename P::Acc acc = P::acc0();
#pragma unroll 8
                for (int c = 0; c < b; ++c) P::fma(acc, P::ld(Gj + (long long)c * b), dj[c]);
                sPhi[t] = P::get(acc);
            }
            __syncthreads();
            // (2.1) publish face data; psi_j for the interior levels
            S* my_mail = mail + q * p.mail_stride + p.mail_off[s];
            for (int t = threadIdx.x; t < kb; t += blockDim.x) {
                const C srcv = (sof >= 0) ? P::mul(P::ld(p.src + sof + t), w) : P::zero();
                if (t < b) P::st(my_mail + t, P::add(sPhi[t], srcv));
                else sD[t] = P::add(P::sub(sPhi[t], sPhi[t - b]), srcv);
            }
            __syncthreads();
            // (2.2) interior update, Eq. (19)
            for (int t = b + threadIdx.x; t < kb; t += blockDim.x) {
                const int j = t / b, i = t - j * b;
                const S* Ghj = Gh + (long long)j * b * b + i;
                const C* pj = sD + j * b;
                typename P::Acc acc = P::acc0();
#pragma unroll 8
                for (int c = 0; c < b; ++c) P::fma(acc, P::ld(Ghj + (long long)c * b), pj[c]);
                const C d = P::add(P::ld(dU + t), P::mul(dt2, P::get(acc)));
                P::st(dU + t, d);
                P::st(Un + t, P::add(sU[t], d));
            }
        }

        if (!grid_barrier(p.bar, (unsigned)(n + 1) * gridDim.x, p.err, p.timeout_ns,
                          p.skip_arrive))
            return;

        // ---------------- phase B: faces, Eq. (18) ----------------
        for (int u = blockIdx.x; u < p.nunits; u += gridDim.x) {
            const int q = u / p.nsub, s = u - q * p.nsub;
            const int b = p.sub_b[s];
            const long long so = q * p.state_stride + p.state_off[s];
            const S* mine = mail + q * p.mail_stride + p.mail_off[s];
            const int* fo = p.face_off + s * 7;
            __syncthreads();
            // sum of both sides' face data, lower subdomain index first
            for (int t = threadIdx.x; t < b; t += blockDim.x) {
                int f = 0;
                while (t >= fo[f + 1]) ++f;
                const int nb = p.nbr[s * 6 + f];
                C v = P::ld(mine + t);
                if (nb >= 0) {
                    const S* other = mail + q * p.mail_stride + p.mail_off[nb];
                    const C o = P::ld(other + p.face_off[nb * 7 + (f ^ 1)] + (t - fo[f]));
                    v = (nb < s) ? P::add(o, v) : P::add(v, o);
                }
                sD[t] = v;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < b; t += blockDim.x) {
                int f = 0;
                while (t >= fo[f + 1]) ++f;
                const int m = fo[f + 1] - fo[f], i = t - fo[f];
                const S* H = p.H + p.H_off[s * 6 + f] + i;   // H symmetric
                const C* v = sD + fo[f];
                typename P::Acc acc = P::acc0();
                for (int c = 0; c < m; ++c) P::fma(acc, P::ld(H + c * m), v[c]);
                const C d = P::add(P::ld(p.dU + so + t), P::mul(dt2, P::get(acc)));
                P::st(p.dU + so + t, d);
                P::st(Unxt + so + t, P::add(P::ld(Ucur + so + t), d));
            }
        }
        // receiver readout of U^n (complete since the barrier above)
        readout<P>(p, Ucur, n, red);
    }
    // final readout of U^{nsteps}, after every face update of the last step
    if (!grid_barrier(p.bar, (unsigned)(p.nsteps + 1) * gridDim.x, p.err, p.timeout_ns,
                      p.skip_arrive))
        return;
    readout<P>(p, p.U[p.nsteps % 3], p.nsteps, red);
}

template <class P>
size_t step_smem_bytes(int kmax, int bmax, int block) {
    (void)block;
    return sizeof(typename P::C) *
           ((size_t)(kmax + 1) * bmax + 2 * (size_t)kmax * bmax + 32);
}

template <class P>
int step_max_grid(int block, size_t smem, int* grid_out) {
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(step_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<P>, block, smem);
    if (per_sm < 1) return -1;
    *grid_out = per_sm * nsm;
    return 0;
}

template <class P>
cudaError_t launch_step(const StepParams<typename P::S>& p, int block, int grid, cudaStream_t st) {
    const size_t smem = step_smem_bytes<P>(p.kmax, p.bmax, block);
    cudaError_t e = cudaFuncSetAttribute(step_kernel<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    StepParams<typename P::S> pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((void*)step_kernel<P>, dim3(grid), dim3(block), args, smem,
                                       st);
}

#define SFM_INST(P)                                                                             \
    template cudaError_t launch_step<P>(const StepParams<P::S>&, int, int, cudaStream_t);       \
    template int step_max_grid<P>(int, size_t, int*);                                           \
    template size_t step_smem_bytes<P>(int, int, int);
SFM_INST(PolF64)
SFM_INST(PolF32)
SFM_INST(PolF32x2)
#undef SFM_INST

// ---------------------------------------------------------------------------
// traces[q][r][n] = sum over the pairs of receiver r of partial[q][n][pair]
// (fixed order, so the result is deterministic).  Flags non-finite values.
template <class P>
__global__ void reduce_traces_kernel(const typename P::S* partial, const int* rec_ptr,
                                     const int* rec_pairs, int nshots, int nsteps, int nrec,
                                     int nrpairs, double* traces, int* bad) {
    const long long total = (long long)nshots * nrec * (nsteps + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i % (nsteps + 1));
        const long long qr = i / (nsteps + 1);
        const int r = (int)(qr % nrec), q = (int)(qr / nrec);
        double acc = 0.0;
        for (int e = rec_ptr[r]; e < rec_ptr[r + 1]; ++e)
            acc += P::to_d(partial[((long long)q * (nsteps + 1) + n) * nrpairs + rec_pairs[e]]);
        traces[i] = acc;
        if (!isfinite(acc)) atomicExch(bad, 1);
    }
}

template <class P>
cudaError_t launch_reduce_traces(const typename P::S* partial, const int* rec_ptr,
                                 const int* rec_pairs, int nshots, int nsteps, int nrec,
                                 int nrpairs, double* traces, int* bad, cudaStream_t st) {
    const long long total = (long long)nshots * nrec * (nsteps + 1);
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    reduce_traces_kernel<P><<<grid, 256, 0, st>>>(partial, rec_ptr, rec_pairs, nshots, nsteps,
                                                  nrec, nrpairs, traces, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <class P>
__global__ void convert_kernel(const double* in, typename P::S* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        P::st(out + i, P::from_d(in[i]));
}

template <class P>
cudaError_t launch_convert(const double* in, typename P::S* out, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    size_t g = (n + 255) / 256;
    int grid = (int)(g > 8192 ? 8192 : g);
    convert_kernel<P><<<grid, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

#define SFM_INST2(P)                                                                           \
    template cudaError_t launch_reduce_traces<P>(const P::S*, const int*, const int*, int, int, \
                                                 int, int, double*, int*, cudaStream_t);       \
    template cudaError_t launch_convert<P>(const double*, P::S*, size_t, cudaStream_t);
SFM_INST2(PolF64)
SFM_INST2(PolF32)
SFM_INST2(PolF32x2)
#undef SFM_INST2

// ---------------------------------------------------------------------------
// Power iteration helpers: sum of squares (one block, fixed order) and the
// normalisation y = x / sqrt(sumsq).
__global__ void sumsq_kernel(const double* x, size_t n, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * x[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) *out = acc;
}

__global__ void scale_kernel(const double* x, double* y, size_t n, const double* sumsq) {
    const double s = 1.0 / sqrt(*sumsq);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}

cudaError_t launch_sumsq(const double* x, size_t n, double* out, cudaStream_t st) {
    sumsq_kernel<<<1, 1024, 0, st>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double* x, double* y, size_t n, const double* sumsq,
                         cudaStream_t st) {
    size_t g = (n + 255) / 256;
    scale_kernel<<<(int)(g > 4096 ? 4096 : (g ? g : 1)), 256, 0, st>>>(x, y, n, sumsq);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Face coupling H_f = (sum over sides of [Gammahat_1]_f^{-1})^{-1}  (Eq. 18),
// FP64, one block per (subdomain, face).  Each side computes its own copy
// with the lower subdomain's term first, so both copies are identical.

// In-place inverse of an SPD m x m matrix (row-major, leading dimension m)
// through its Cholesky factor; returns false on a non-positive pivot.
__device__ bool spd_inverse_serial(double* A, int m, double* L) {
    for (int i = 0; i < m * m; ++i) L[i] = 0.0;
    for (int j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int c = 0; c < j; ++c) d -= L[j * m + c] * L[j * m + c];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        L[j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double v = A[i * m + j];
            for (int c = 0; c < j; ++c) v -= L[i * m + c] * L[j * m + c];
            L[i * m + j] = v / d;
        }
    }
    // A = L^{-T} L^{-1}: first invert L in place (lower triangular)
    for (int j = 0; j < m; ++j) {
        L[j * m + j] = 1.0 / L[j * m + j];
        for (int i = j + 1; i < m; ++i) {
            double v = 0.0;
            for (int c = j; c < i; ++c) v -= L[i * m + c] * L[c * m + j];
            L[i * m + j] = v / L[i * m + i];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int c = i; c < m; ++c) v += L[c * m + i] * L[c * m + j];
            A[i * m + j] = v;
            A[j * m + i] = v;
        }
    return true;
}

__global__ void face_H_kernel(const double* coef, const long long* gh1_off, const int* sub_b,
                              const int* face_off, const int* nbr, const long long* H_off,
                              double* H, int nsub, int* err) {
    __shared__ double A[SFM_MAX_FACE_M * SFM_MAX_FACE_M];
    __shared__ double B[SFM_MAX_FACE_M * SFM_MAX_FACE_M];
    __shared__ double W[SFM_MAX_FACE_M * SFM_MAX_FACE_M];
    const int sf = blockIdx.x;
    const int s = sf / 6, f = sf % 6;
    if (s >= nsub || threadIdx.x != 0) return;
    const int m = face_off[s * 7 + f + 1] - face_off[s * 7 + f];
    if (m == 0) return;
    const int nb = nbr[s * 6 + f];
    // the lower-numbered side's term first
    const int lo = (nb >= 0 && nb < s) ? nb : s;
    const int hi = (nb >= 0 && nb < s) ? s : nb;
    const int flo = (lo == s) ? f : (f ^ 1);
    const int fhi = (hi == s) ? f : (f ^ 1);
    {
        const int bt = sub_b[lo];
        const double* G = coef + gh1_off[lo];
        const int o = face_off[lo * 7 + flo];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) A[i * m + j] = G[(long long)(o + i) * bt + (o + j)];
        if (!spd_inverse_serial(A, m, W)) { atomicCAS(err, 0, (int)SFM_ERR_NOT_SPD); return; }
    }
    if (nb >= 0) {
        const int bt = sub_b[hi];
        const double* G = coef + gh1_off[hi];
        const int o = face_off[hi * 7 + fhi];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) B[i * m + j] = G[(long long)(o + i) * bt + (o + j)];
        if (!spd_inverse_serial(B, m, W)) { atomicCAS(err, 0, (int)SFM_ERR_NOT_SPD); return; }
        for (int i = 0; i < m * m; ++i) A[i] = A[i] + B[i];
    }
    if (!spd_inverse_serial(A, m, W)) { atomicCAS(err, 0, (int)SFM_ERR_NOT_SPD); return; }
    double* out = H + H_off[s * 6 + f];
    for (int i = 0; i < m * m; ++i) out[i] = A[i];
}

cudaError_t launch_face_H(const double* coef, const long long* gh1_off, const int* sub_b,
                          const int* face_off, const int* nbr, const long long* H_off, double* H,
                          int nsub, int* err, cudaStream_t st) {
    face_H_kernel<<<nsub * 6, 32, 0, st>>>(coef, gh1_off, sub_b, face_off, nbr, H_off, H, nsub,
                                           err);
    return cudaGetLastError();
}

}  // namespace sfm
