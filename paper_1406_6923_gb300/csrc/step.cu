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

// y = M x for a symmetric b x b block M stored as its upper triangle of 8x8
// tiles (tile (I,J), J >= I, at index I*nt - I(I-1)/2 + (J-I), row-major
// inside the tile); one warp per block.  Lane (r, q) accumulates row 8I+r
// over columns 8J+2q, 8J+2q+1 of every tile column J: a stored tile is one
// coalesced 16-byte load per lane, a tile below the diagonal is read
// transposed from its stored mirror (the same warp just touched it, so it
// comes from L1).  x and y are in shared memory, padded to 8*nt.
constexpr int NTMAX = 8;   // b <= 64

template <class P>
__device__ __forceinline__ void warp_symv(const typename P::S* tiles, int nt,
                                          const typename P::C* x, typename P::C* y) {
    using C = typename P::C;
    const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
    for (int I = 0; I < nt; ++I) {
        C e0[NTMAX], e1[NTMAX];
#pragma unroll
        for (int J = 0; J < NTMAX; ++J) {
            if (J < nt) {
                if (J >= I) {
                    P::ld2(tiles + (long long)(I * nt - I * (I - 1) / 2 + (J - I)) * 64 + r * 8 + 2 * q,
                           e0[J], e1[J]);
                } else {
                    const typename P::S* t = tiles + (long long)(J * nt - J * (J - 1) / 2 + (I - J)) * 64;
                    e0[J] = P::ldg(t + (2 * q) * 8 + r);
                    e1[J] = P::ldg(t + (2 * q + 1) * 8 + r);
                }
            }
        }
        typename P::Acc acc = P::acc0();
#pragma unroll
        for (int J = 0; J < NTMAX; ++J) {
            if (J < nt) {
                P::fma(acc, e0[J], x[8 * J + 2 * q]);
                P::fma(acc, e1[J], x[8 * J + 2 * q + 1]);
            }
        }
        C v = P::get(acc);
        v = P::add(v, P::shfl_xor(v, 1));
        v = P::add(v, P::shfl_xor(v, 2));
        if (q == 0) y[8 * I + r] = v;
    }
}

template <class P>
__global__ void __launch_bounds__(256) step_kernel(StepParams<typename P::S> p) {
    using S = typename P::S;
    using C = typename P::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bpm = ((p.bmax + 7) / 8) * 8;              // padded block width
    C* sU = reinterpret_cast<C*>(smem_raw);              // (kmax+1)*bpm
    C* sD = sU + (p.kmax + 1) * bpm;                     // kmax*bpm: Delta, then psi
    C* sPhi = sD + p.kmax * bpm;                         // kmax*bpm: phi, then a
    C* red = sPhi + p.kmax * bpm;                        // 32
    const C dt2 = P::from_d(p.dt2);

    for (int n = 0; n < p.nsteps; ++n) {
        const S* Ucur = p.U[n % 3];
        S* Unxt = p.U[(n + 1) % 3];
        S* mail = (n & 1) ? p.mail1 : p.mail0;

        // ---------------- phase A ----------------
        for (int u = blockIdx.x; u < p.nunits; u += gridDim.x) {
            const int q = u / p.nsub, s = u - q * p.nsub;
            const int b = p.sub_b[s], k = p.sub_k[s], kb = k * b;
            const int nt = (b + 7) >> 3, bp = nt * 8;
            const long long ltile = 2LL * (nt * (nt + 1) / 2) * 64;   // per level
            const long long so = q * p.state_stride + p.state_off[s];
            const S* Uc = Ucur + so;
            S* Un = Unxt + so;
            S* dU = p.dU + so;
            const S* T0 = p.coef + p.coef_off[s];   // level j: Gamma_j at T0 + j*ltile,
                                                    // Gammahat_j at T0 + j*ltile + ltile/2
            const long long sof = p.src_off[(long long)q * p.nsub + s];
            const C w = P::ld(p.wavelet + (long long)q * p.nsteps + n);
            const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
            __syncthreads();
            // padded copies: level j occupies [j*bp, j*bp + b), zeros up to bp
            for (int t = threadIdx.x; t < (k + 1) * bp; t += blockDim.x) {
                const int j = t / bp, i = t - j * bp;
                sU[t] = (j < k && i < b) ? P::ld(Uc + j * b + i) : P::zero();
            }
            __syncthreads();
            for (int t = threadIdx.x; t < k * bp; t += blockDim.x) sD[t] = P::sub(sU[t + bp], sU[t]);
            __syncthreads();
            // phi_j = Gamma_j Delta_j, j = 1..k: one warp per level
            for (int j = warp; j < k; j += nwarp)
                warp_symv<P>(T0 + (long long)j * ltile, nt, sD + j * bp, sPhi + j * bp);
            __syncthreads();
            // (2.1) publish face data; psi_j for the interior levels
            S* my_mail = mail + q * p.mail_stride + p.mail_off[s];
            for (int t = threadIdx.x; t < kb; t += blockDim.x) {
                const int j = t / b, i = t - j * b;
                const C srcv = (sof >= 0) ? P::mul(P::ld(p.src + sof + t), w) : P::zero();
                if (j == 0) P::st(my_mail + i, P::add(sPhi[i], srcv));
                else sD[j * bp + i] = P::add(P::sub(sPhi[j * bp + i], sPhi[(j - 1) * bp + i]), srcv);
            }
            __syncthreads();
            // (2.2) a_j = Gammahat_j psi_j for j >= 2 (into sPhi), Eq. (19)
            for (int j = 1 + warp; j < k; j += nwarp)
                warp_symv<P>(T0 + (long long)j * ltile + ltile / 2, nt, sD + j * bp, sPhi + j * bp);
            __syncthreads();
            if (p.Kx)
                for (int t = b + threadIdx.x; t < kb; t += blockDim.x)
                    P::st(p.Kx + so + t, sD[(t / b) * bp + (t % b)]);
            for (int t = b + threadIdx.x; t < kb; t += blockDim.x) {
                const int j = t / b, i = t - j * b;
                const C d = P::add(P::ld(dU + t), P::mul(dt2, sPhi[j * bp + i]));
                P::st(dU + t, d);
                P::st(Un + t, P::add(sU[j * bp + i], d));
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
                if (p.Kx) P::st(p.Kx + so + t, v);
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
    const size_t bp = (size_t)((bmax + 7) / 8) * 8;
    return sizeof(typename P::C) * ((size_t)(kmax + 1) * bp + 2 * (size_t)kmax * bp + 32);
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

template <class P>
__global__ void pack_tiles_kernel(const double* master, const long long* master_off,
                                  const long long* tile_off, const int* sub_b, const int* sub_k,
                                  typename P::S* out) {
    const int s = blockIdx.y;
    const int b = sub_b[s], k = sub_k[s];
    const int nt = (b + 7) / 8, T = nt * (nt + 1) / 2;
    const long long total = 2LL * k * T * 64;
    const double* m = master + master_off[s];
    typename P::S* o = out + tile_off[s];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int rc = (int)(e & 63);
        long long rest = e >> 6;
        const int tix = (int)(rest % T);
        rest /= T;
        const int which = (int)(rest & 1), j = (int)(rest >> 1);
        int I = 0, base = 0;
        while (base + (nt - I) <= tix) { base += nt - I; ++I; }
        const int J = I + (tix - base);
        const int row = 8 * I + (rc >> 3), col = 8 * J + (rc & 7);
        double v = 0.0;
        if (row < b && col < b) v = m[((long long)which * k + j) * b * b + (long long)row * b + col];
        P::st(o + e, P::from_d(v));
    }
}

template <class P>
cudaError_t launch_pack_tiles(const double* master, const long long* master_off,
                              const long long* tile_off, const int* sub_b, const int* sub_k,
                              int nsub, typename P::S* out, cudaStream_t st) {
    for (int s0 = 0; s0 < nsub; s0 += 65535) {
        const int ns = nsub - s0 < 65535 ? nsub - s0 : 65535;
        pack_tiles_kernel<P><<<dim3(64, ns), 256, 0, st>>>(master, master_off + s0, tile_off + s0,
                                                          sub_b + s0, sub_k + s0, out);
    }
    return cudaGetLastError();
}

#define SFM_INST2(P)                                                                           \
    template cudaError_t launch_reduce_traces<P>(const P::S*, const int*, const int*, int, int, \
                                                 int, int, double*, int*, cudaStream_t);       \
    template cudaError_t launch_convert<P>(const double*, P::S*, size_t, cudaStream_t);        \
    template cudaError_t launch_pack_tiles<P>(const double*, const long long*, const long long*, \
                                              const int*, const int*, int, P::S*, cudaStream_t);
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

__global__ void wdot_kernel(const double* x, const double* y, const double* w, size_t n,
                            double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) acc += w[i] * x[i] * y[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) *out = acc;
}

cudaError_t launch_wdot(const double* x, const double* y, const double* w, size_t n, double* out,
                        cudaStream_t st) {
    wdot_kernel<<<1, 1024, 0, st>>>(x, y, w, n, out);
    return cudaGetLastError();
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
