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
//   the receiver readout of U^n runs inside the next step's barrier, between
//   this block's arrival and its wait, taken item by item from a counter
//
// Each subdomain keeps its own copy of its level-1 face blocks; both sides
// of a shared face compute the same sum of the same two mail vectors with
// the same H_f copy, so the two copies stay bitwise equal (the continuity
// condition of Eq. 17).  U^n lives in buffer n % 4 and the mail in buffer
// n % 2: a block that runs ahead into phase A of step n+1 then never writes
// what a slower block still reads in phase B of step n or in the readout,
// so one barrier per step suffices.
#include "sfm_internal.h"
#include "step_kernel.cuh"

#include <cooperative_groups.h>
#include <climits>
#include <algorithm>

namespace sfm {

// Pieces of work per block: the (unit, level) sequence, unit-major, cut into
// contiguous pieces, one list per block, so that the blocks' estimated costs
// are as even as a greedy fill allows.  Cost unit: one level (its two block
// products); a block's second and later pieces add their staging and
// barriers, a level-0 piece adds the face data and the face update, and a
// piece starting at level >= 2 recomputes phi_{j0-1}.  The smallest
// capacity whose greedy fill needs at most `grid` blocks is found by
// bisection.  A unit is never cut at level 1: a piece starting there would
// read the level-0 face blocks, which the level-0 piece updates after the
// device-wide barrier, with no barrier before the next step's phase A;
// pieces starting at level >= 2 read only interior levels, which are
// written before the barrier.
void build_pieces(int nunits, int nsub, const int* k_sub, int grid, std::vector<int>& ptr,
                  std::vector<int4>& pieces) {
    const double kPiece = 2.0, kFace = 2.0, kLead = 0.5;
    long long total = 0;
    int kmax = 1;
    for (int u = 0; u < nunits; ++u) {
        total += k_sub[u % nsub];
        kmax = std::max(kmax, k_sub[u % nsub]);
    }
    auto fill = [&](double cap, bool emit) -> int {
        if (emit) { ptr.assign(grid + 1, 0); pieces.clear(); }
        int blocks = 0, u = 0, j = 0;
        while (u < nunits) {
            if (emit) {
                if (blocks >= grid) return blocks + 1;
                ptr[blocks] = (int)pieces.size();
            }
            ++blocks;
            double used = 0.0;
            int np = 0;
            while (u < nunits) {
                const int k = k_sub[u % nsub];
                const double over = (np > 0 ? kPiece : 0.0) + (j == 0 ? kFace : 0.0) + (j >= 2 ? kLead : 0.0);
                int take = (int)std::min<double>(k - j, std::floor(cap - used - over));
                if (j + take == 1 && k > 1) take = (cap - used - over >= 2.0) ? 2 : 0;   // no cut at level 1
                if (take <= 0 && np == 0) take = (j == 0 && k > 1) ? 2 : 1;             // always progress
                if (take <= 0) break;
                if (emit) pieces.push_back(make_int4(u, j, j + take, 0));
                used += over + take;
                ++np;
                j += take;
                const bool whole = (j == k);
                if (whole) { ++u; j = 0; }
                if (!whole) break;                                                     // block full
            }
        }
        if (emit)
            for (int c = blocks; c <= grid; ++c) ptr[c] = (int)pieces.size();
        return blocks;
    };
    double lo = (double)total / grid, hi = lo + kmax + 4 * (kPiece + kFace + kLead) + 2;
    while (fill(hi, false) > grid) hi *= 2;
    for (int it = 0; it < 40 && hi - lo > 1e-3; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (fill(mid, false) <= grid) hi = mid; else lo = mid;
    }
    fill(hi, true);
}

// Piece records, two int4 per piece: {shot, subdomain, j0, j1} and
// {b | k << 8, state offset, source-row offset (with the shot, -1 if none),
// face-data offset}.  False if an offset does not fit in 32 bits.
bool piece_records(const std::vector<int4>& pieces, int nsub, const int* k, const int* b,
                   const long long* state_off, const long long* src_off, const long long* mail_off,
                   std::vector<int4>& rec) {
    rec.resize(2 * pieces.size());
    for (size_t i = 0; i < pieces.size(); ++i) {
        const int u = pieces[i].x, q = u / nsub, s = u - q * nsub;
        const long long sof = src_off[(size_t)q * nsub + s];
        if (state_off[s] > INT_MAX || sof > INT_MAX || mail_off[s] > INT_MAX || b[s] > 255)
            return false;
        rec[2 * i] = make_int4(q, s, pieces[i].y, pieces[i].z);
        rec[2 * i + 1] = make_int4(b[s] | (k[s] << 8), (int)state_off[s], (int)sof, (int)mail_off[s]);
    }
    return true;
}

// Per-row face table in the layout of the face data (row mail_off[s] + t):
// {neighbour's face-data offset of the same face node (-1 on an outer face),
//  offset of row i of H_f, m_f | (neighbour index < s) << 16, start of the
//  face inside the b-vector}.
bool face_rows(int nsub, const int* b, const int* face_off, const int* nbr,
               const long long* H_off, const long long* mail_off, std::vector<int4>& rows) {
    long long n = 0;
    for (int s = 0; s < nsub; ++s) n += b[s];
    rows.assign((size_t)n, make_int4(-1, 0, 0, 0));
    for (int s = 0; s < nsub; ++s) {
        for (int f = 0; f < 6; ++f) {
            const int f0 = face_off[s * 7 + f], m = face_off[s * 7 + f + 1] - f0;
            const int nb = nbr[s * 6 + f];
            for (int i = 0; i < m; ++i) {
                long long other = -1;
                if (nb >= 0) other = mail_off[nb] + face_off[nb * 7 + (f ^ 1)] + i;
                const long long h = H_off[s * 6 + f] + i;
                if (other > INT_MAX || h > INT_MAX || mail_off[s] + f0 + i > INT_MAX) return false;
                rows[(size_t)(mail_off[s] + f0 + i)] =
                    make_int4((int)other, (int)h, m | ((nb >= 0 && nb < s) ? 1 << 16 : 0), f0);
            }
        }
    }
    return true;
}

// Receiver pair table: {k*b of its subdomain, row offset, state offset, 0}.
bool readout_table(int nrpairs, const int* rp_sub, const long long* rp_off, const int* k,
                   const int* b, const long long* state_off, std::vector<int4>& tab) {
    tab.resize((size_t)std::max(nrpairs, 1), make_int4(0, 0, 0, 0));
    for (int r = 0; r < nrpairs; ++r) {
        const int s = rp_sub[r];
        if (rp_off[r] > INT_MAX || state_off[s] > INT_MAX) return false;
        tab[r] = make_int4(k[s] * b[s], (int)rp_off[r], (int)state_off[s], 0);
    }
    return true;
}

#define SFM_INST(P)                                                                             \
    template cudaError_t launch_step<P>(const StepParams<P::S>&, int, cudaStream_t);            \
    template int step_max_grid<P>(int, size_t, int*);                                           \
    template size_t step_smem_bytes<P>(int, int, int);
SFM_INST(PolF64)
SFM_INST(PolF32)
SFM_INST(PolF32x2)
SFM_INST(PolF32F)
SFM_INST(PolF32Fx2)
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

// Cholesky factors of the S-fraction blocks for the factored FP32 policy.
// One block of threads per (subdomain, coefficient block): Gamma_j is block
// 2j, Gammahat_j block 2j+1 (the level-major order of the packed tiles).
// The b x b FP64 block is factored in shared memory (right-looking, column
// by column, in FP64), then rounded to FP32 into lower-triangular 8x8 tiles.
// A non-positive pivot down to -1e-8 max|diag| (rounding in a block that is
// singular) is a semi-definite direction: its column of the factor is
// zero.  A pivot below that in a block the stepping
// uses (every Gamma_j and Gammahat_j for j >= 2) sets *bad; Gammahat_1 is
// replaced by H_f on the faces and is not needed.
constexpr int FAC_LD = 65;

__global__ void __launch_bounds__(256) factor_tiles_kernel(const double* master,
                                                           const long long* master_off,
                                                           const long long* tile_off,
                                                           const int* sub_b, const int* sub_k,
                                                           float* out, int* bad) {
    __shared__ double A[64 * FAC_LD];
    const int s = blockIdx.y, blk = blockIdx.x;
    const int b = sub_b[s], k = sub_k[s];
    if (blk >= 2 * k) return;
    const int j = blk >> 1, which = blk & 1;
    const int nt = (b + 7) / 8, T = nt * (nt + 1) / 2;
    const double* m = master + master_off[s] + ((long long)which * k + j) * b * b;
    __shared__ double s_scale;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) A[(e / b) * FAC_LD + e % b] = m[e];
    __syncthreads();
    if (threadIdx.x == 0) {
        double sc = 0.0;
        for (int i = 0; i < b; ++i) sc = fmax(sc, fabs(A[i * FAC_LD + i]));
        s_scale = sc;
    }
    bool ok = true;
    for (int c = 0; c < b; ++c) {
        __syncthreads();
        const double d = A[c * FAC_LD + c];     // same value in every thread
        if (!(d > 0.0)) {
            // a semi-definite block (singular to rounding): zero pivot, zero
            // column; a clearly negative pivot means the block is indefinite
            if (!(d >= -1e-8 * s_scale)) { ok = false; break; }
            __syncthreads();
            for (int i = c + threadIdx.x; i < b; i += blockDim.x) A[i * FAC_LD + c] = 0.0;
            continue;
        }
        const double l = sqrt(d);
        __syncthreads();
        if (threadIdx.x == 0) A[c * FAC_LD + c] = l;
        for (int i = c + 1 + threadIdx.x; i < b; i += blockDim.x) A[i * FAC_LD + c] /= l;
        __syncthreads();
        const int n = b - c - 1;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = c + 1 + t / n, jj = c + 1 + t % n;
            if (jj <= i) A[i * FAC_LD + jj] -= A[i * FAC_LD + c] * A[jj * FAC_LD + c];
        }
    }
    __syncthreads();
    if (!ok) {
        if (threadIdx.x == 0 && !(which == 1 && j == 0)) atomicExch(bad, 1);
    }
    float* o = out + tile_off[s] + (long long)blk * T * 64;
    for (int e = threadIdx.x; e < T * 64; e += blockDim.x) {
        const int tix = e >> 6, rc = e & 63;
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= tix) ++I;
        const int J = tix - I * (I + 1) / 2;
        const int row = 8 * I + (rc >> 3), col = 8 * J + (rc & 7);
        const double v = (ok && row < b && col <= row) ? A[row * FAC_LD + col] : 0.0;
        o[e] = __double2float_rn(v);
    }
}

cudaError_t launch_factor_tiles(const double* master, const long long* master_off,
                                const long long* tile_off, const int* sub_b, const int* sub_k,
                                int nsub, int kmax, float* out, int* bad, cudaStream_t st) {
    for (int s0 = 0; s0 < nsub; s0 += 65535) {
        const int ns = nsub - s0 < 65535 ? nsub - s0 : 65535;
        factor_tiles_kernel<<<dim3(2 * kmax, ns), 256, 0, st>>>(master, master_off + s0,
                                                                tile_off + s0, sub_b + s0,
                                                                sub_k + s0, out, bad);
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
SFM_INST2(PolF32F)
SFM_INST2(PolF32Fx2)
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

// Starting increment of the initial-value form: delta^0 = dt V^0 - dt^2/2 a.
__global__ void start_delta_kernel(const double* v, const double* a, double dt, size_t n,
                                   double* out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (v ? dt * v[i] : 0.0) - 0.5 * dt * dt * a[i];
}

cudaError_t launch_start_delta(const double* v, const double* a, double dt, size_t n, double* out,
                               cudaStream_t st) {
    size_t g = (n + 255) / 256;
    start_delta_kernel<<<(int)(g > 4096 ? 4096 : (g ? g : 1)), 256, 0, st>>>(v, a, dt, n, out);
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
