// Device kernels of the FP64 offline ROM builder (Algorithm 1 stage 1).
//
// Fine operator (the reading of Eq. 1 used throughout the library): vertex-
// centred finite volumes on cubic cells of side h.  Every cell adds h/4 to
// the conductance of each of its 12 edges and h^3/(8 c^2) to the lumped mass
// of each of its 8 corner nodes.  Inside a subdomain box of nx*ny*nz cells an
// x-edge between nodes (i,j,k) and (i+1,j,k) therefore has conductance
// (h/4) w_y(j) w_z(k), with w(j) = 1 on the box boundary and 2 inside; the
// box boundary is natural (homogeneous Neumann).  L = M^{-1/2} K M^{-1/2}.
#pragma once

#include <cuda_runtime.h>

namespace sfm {
namespace bld {

// ---------------------------------------------------------------------------
// lumped mass of every node of every subdomain of a class
__global__ void mass_kernel(const double* c, int gnx, int gny, const int3* origin, int S,
                            int nxl, int nyl, int nzl, double h, double* mass) {
    const int N = (nxl + 1) * (nyl + 1) * (nzl + 1);
    const long long total = (long long)S * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / N), n = (int)(t % N);
        const int i = n % (nxl + 1), j = (n / (nxl + 1)) % (nyl + 1), k = n / ((nxl + 1) * (nyl + 1));
        const int3 o = origin[s];
        double m = 0.0;
        for (int dk = -1; dk <= 0; ++dk) {
            const int ck = k + dk;
            if (ck < 0 || ck >= nzl) continue;
            for (int dj = -1; dj <= 0; ++dj) {
                const int cj = j + dj;
                if (cj < 0 || cj >= nyl) continue;
                for (int di = -1; di <= 0; ++di) {
                    const int ci = i + di;
                    if (ci < 0 || ci >= nxl) continue;
                    const double v = c[((long long)(o.z + ck) * gny + (o.y + cj)) * gnx + (o.x + ci)];
                    m += h * h * h / (8.0 * v * v);
                }
            }
        }
        mass[t] = m;
    }
}

// Face basis B (N x b, column-major) of a class: column col is mode (p,q) of
// face f on the open face, h^2 cos(pi p (s-1/2)/ns) cos(pi q (t-1/2)/nt).
struct ColSpec {
    int f, p, q, pad;
};

__global__ void basis_kernel(const ColSpec* cols, int b, int nxl, int nyl, int nzl, double h,
                             double* B) {
    const int N = (nxl + 1) * (nyl + 1) * (nzl + 1);
    const int ncell[3] = {nxl, nyl, nzl};
    const long long total = (long long)N * b;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(t / N), n = (int)(t % N);
        const int g[3] = {n % (nxl + 1), (n / (nxl + 1)) % (nyl + 1), n / ((nxl + 1) * (nyl + 1))};
        const ColSpec cs = cols[col];
        const int a = cs.f >> 1;
        const int u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2;
        double val = 0.0;
        const bool on_face = (cs.f & 1) ? (g[a] == ncell[a]) : (g[a] == 0);
        const int s_ = g[u], t_ = g[v];
        if (on_face && s_ > 0 && s_ < ncell[u] && t_ > 0 && t_ < ncell[v]) {
            const int ns = ncell[u] - 1, nt = ncell[v] - 1;
            val = h * h * cospi((double)cs.p * (s_ - 0.5) / ns) * cospi((double)cs.q * (t_ - 0.5) / nt);
        }
        B[t] = val;
    }
}

// Y[s][col][n] = X[s or shared][col][n] * mass[s][n]^power  (power = +-1/2)
__global__ void scale_kernel(const double* X, long long sX, const double* mass, double* Y,
                             long long sY, int N, int ncol, int S, int inverse) {
    const long long total = (long long)S * ncol * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(t % N);
        const long long sc = t / N;
        const int col = (int)(sc % ncol), s = (int)(sc / ncol);
        const double m = sqrt(mass[(long long)s * N + n]);
        const double x = X[s * sX + (long long)col * N + n];
        Y[s * sY + (long long)col * N + n] = inverse ? x / m : x * m;
    }
}

// ---------------------------------------------------------------------------
// Shifted operator (K + sigma M) applied to one column per block, with the
// column's dot product x.y.  Columns are N-long and contiguous; column
// `gc` = s * ncol + col belongs to subdomain s.
__device__ __forceinline__ double edge_w(int j, int n) { return (j == 0 || j == n) ? 1.0 : 2.0; }

__device__ __forceinline__ double block_reduce_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

__device__ __forceinline__ double apply_row(const double* x, int i, int j, int k, int nxl, int nyl,
                                            int nzl, double q4, double diag_shift) {
    const int sx = 1, sy = nxl + 1, sz = (nxl + 1) * (nyl + 1);
    const int n = i + sy * j + sz * k;
    const double xc = x[n];
    double acc = diag_shift * xc;
    const double wy = edge_w(j, nyl), wz = edge_w(k, nzl), wx = edge_w(i, nxl);
    if (i > 0) acc += q4 * wy * wz * (xc - x[n - sx]);
    if (i < nxl) acc += q4 * wy * wz * (xc - x[n + sx]);
    if (j > 0) acc += q4 * wx * wz * (xc - x[n - sy]);
    if (j < nyl) acc += q4 * wx * wz * (xc - x[n + sy]);
    if (k > 0) acc += q4 * wx * wy * (xc - x[n - sz]);
    if (k < nzl) acc += q4 * wx * wy * (xc - x[n + sz]);
    return acc;
}

__device__ __forceinline__ double diag_of(int i, int j, int k, int nxl, int nyl, int nzl, double q4) {
    const double wx = edge_w(i, nxl), wy = edge_w(j, nyl), wz = edge_w(k, nzl);
    double d = 0.0;
    d += ((i > 0) + (i < nxl)) * q4 * wy * wz;
    d += ((j > 0) + (j < nyl)) * q4 * wx * wz;
    d += ((k > 0) + (k < nzl)) * q4 * wx * wy;
    return d;
}

// Y = (K + sigma M) X  (scale_io: X and Y in the symmetrised variables, i.e.
// Y = M^{-1/2} (K + sigma M) M^{-1/2} X), and dots[gc] = X . Y
__global__ void __launch_bounds__(256) op_kernel(const double* X, double* Y, const double* mass,
                                                 int nxl, int nyl, int nzl, double h, double sigma,
                                                 int ncol, int scale_io, double* dots) {
    __shared__ double red[32];
    const int N = (nxl + 1) * (nyl + 1) * (nzl + 1);
    const long long gc = blockIdx.x;
    const int s = (int)(gc / ncol);
    const double* x = X + gc * N;
    double* y = Y + gc * N;
    const double* m = mass + (long long)s * N;
    const double q4 = 0.25 * h;
    double acc = 0.0;
    if (!scale_io) {
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            const int i = n % (nxl + 1), j = (n / (nxl + 1)) % (nyl + 1), k = n / ((nxl + 1) * (nyl + 1));
            const double v = apply_row(x, i, j, k, nxl, nyl, nzl, q4, sigma * m[n]);
            y[n] = v;
            acc += x[n] * v;
        }
    } else {
        // symmetrised: y_n = m_n^{-1/2} sum_e g_e (x_n/sqrt(m_n) - x_nb/sqrt(m_nb)) + sigma x_n
        const int sx = 1, sy = nxl + 1, sz = (nxl + 1) * (nyl + 1);
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            const int i = n % (nxl + 1), j = (n / (nxl + 1)) % (nyl + 1), k = n / ((nxl + 1) * (nyl + 1));
            const double wx = edge_w(i, nxl), wy = edge_w(j, nyl), wz = edge_w(k, nzl);
            const double xc = x[n] / sqrt(m[n]);
            double a = 0.0;
            if (i > 0) a += q4 * wy * wz * (xc - x[n - sx] / sqrt(m[n - sx]));
            if (i < nxl) a += q4 * wy * wz * (xc - x[n + sx] / sqrt(m[n + sx]));
            if (j > 0) a += q4 * wx * wz * (xc - x[n - sy] / sqrt(m[n - sy]));
            if (j < nyl) a += q4 * wx * wz * (xc - x[n + sy] / sqrt(m[n + sy]));
            if (k > 0) a += q4 * wx * wy * (xc - x[n - sz] / sqrt(m[n - sz]));
            if (k < nzl) a += q4 * wx * wy * (xc - x[n + sz] / sqrt(m[n + sz]));
            const double v = a / sqrt(m[n]) + sigma * x[n];
            y[n] = v;
            acc += x[n] * v;
        }
    }
    if (dots) {
        acc = block_reduce_d(acc, red);
        if (threadIdx.x == 0) dots[gc] = acc;
    }
}

// Jacobi-preconditioned CG pieces for (K + sigma M) Y = R, one block per column.
// init: X = 0, R = rhs, Z = R / diag, P = Z, rz = R.Z, rr0 = R.R
__global__ void __launch_bounds__(256) cg_init_kernel(const double* rhs, double* X, double* R,
                                                      double* Z, double* P, const double* mass,
                                                      int nxl, int nyl, int nzl, double h,
                                                      double sigma, int ncol, double* rz,
                                                      double* rr0) {
    __shared__ double red[32];
    const int N = (nxl + 1) * (nyl + 1) * (nzl + 1);
    const long long gc = blockIdx.x;
    const int s = (int)(gc / ncol);
    const double* m = mass + (long long)s * N;
    const double q4 = 0.25 * h;
    double a = 0.0, c = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int i = n % (nxl + 1), j = (n / (nxl + 1)) % (nyl + 1), k = n / ((nxl + 1) * (nyl + 1));
        const double d = diag_of(i, j, k, nxl, nyl, nzl, q4) + sigma * m[n];
        const double r = rhs[gc * N + n];
        const double z = r / d;
        X[gc * N + n] = 0.0;
        R[gc * N + n] = r;
        Z[gc * N + n] = z;
        P[gc * N + n] = z;
        a += r * z;
        c += r * r;
    }
    a = block_reduce_d(a, red);
    __syncthreads();
    c = block_reduce_d(c, red);
    if (threadIdx.x == 0) { rz[gc] = a; rr0[gc] = c; }
}

// alpha = rz/pq; X += alpha P; R -= alpha Q; Z = R/diag; rznew = R.Z; rr = R.R
__global__ void __launch_bounds__(256) cg_update_kernel(double* X, double* R, double* Z,
                                                        const double* P, const double* Q,
                                                        const double* mass, int nxl, int nyl,
                                                        int nzl, double h, double sigma, int ncol,
                                                        const double* rz, const double* pq,
                                                        double* rznew, double* rr) {
    __shared__ double red[32];
    const int N = (nxl + 1) * (nyl + 1) * (nzl + 1);
    const long long gc = blockIdx.x;
    const int s = (int)(gc / ncol);
    const double* m = mass + (long long)s * N;
    const double q4 = 0.25 * h;
    const double alpha = (pq[gc] != 0.0) ? rz[gc] / pq[gc] : 0.0;
    double a = 0.0, c = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int i = n % (nxl + 1), j = (n / (nxl + 1)) % (nyl + 1), k = n / ((nxl + 1) * (nyl + 1));
        const long long o = gc * N + n;
        X[o] += alpha * P[o];
        const double r = R[o] - alpha * Q[o];
        R[o] = r;
        const double z = r / (diag_of(i, j, k, nxl, nyl, nzl, q4) + sigma * m[n]);
        Z[o] = z;
        a += r * z;
        c += r * r;
    }
    a = block_reduce_d(a, red);
    __syncthreads();
    c = block_reduce_d(c, red);
    if (threadIdx.x == 0) { rznew[gc] = a; rr[gc] = c; }
}

// P = Z + beta P with beta = rznew/rz; then rz = rznew
__global__ void cg_dir_kernel(double* P, const double* Z, int N, double* rz, const double* rznew) {
    const long long gc = blockIdx.x;
    const double beta = (rz[gc] != 0.0) ? rznew[gc] / rz[gc] : 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const long long o = gc * N + n;
        P[o] = Z[o] + beta * P[o];
    }
    __syncthreads();
    if (threadIdx.x == 0) rz[gc] = rznew[gc];
}

// ---------------------------------------------------------------------------
// Small dense factorisations, one block per matrix (column-major, ld = n).
//
// chol_rinv: A = R^T R (R upper), writes R and R^{-1}; ratio[s] = min diag(R)
// / max diag(R); err on a non-positive pivot.  The work space (2 n*n) is the
// block's dynamic shared memory, or, for blocks too wide for it, its slice
// of the global array ws.
__global__ void chol_rinv_kernel(const double* A, double* Rout, double* Rinv, int n, int* err,
                                 double* ratio, double* ws) {
    extern __shared__ double sm_dyn[];
    double* sm = ws ? ws + (long long)blockIdx.x * 2 * n * n : sm_dyn;
    double* a = sm;            // n*n, column-major: a[i + n*j]
    double* ri = sm + n * n;   // n*n
    const long long s = blockIdx.x;
    const double* As = A + s * n * n;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) { a[t] = As[t]; ri[t] = 0.0; }
    __syncthreads();
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    // upper Cholesky by rows: a becomes R in its upper triangle
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const double d = a[j + n * j];
            if (!(d > 0.0)) bad = 1;
            a[j + n * j] = sqrt(d > 0.0 ? d : 1.0);
        }
        __syncthreads();
        const double djj = a[j + n * j];
        for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) a[j + n * c] /= djj;
        __syncthreads();
        for (int t = threadIdx.x; t < (n - j - 1) * (n - j - 1); t += blockDim.x) {
            const int r = j + 1 + t % (n - j - 1), c = j + 1 + t / (n - j - 1);
            if (r <= c) a[r + n * c] -= a[j + n * r] * a[j + n * c];
        }
        __syncthreads();
    }
    // R^{-1} (upper): column c solves R x = e_c by back substitution
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        for (int r = c; r >= 0; --r) {
            double v = (r == c) ? 1.0 : 0.0;
            for (int l = r + 1; l <= c; ++l) v -= a[r + n * l] * ri[l + n * c];
            ri[r + n * c] = v / a[r + n * r];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int r = t % n, c = t / n;
        Rout[s * n * n + t] = (r <= c) ? a[t] : 0.0;
        Rinv[s * n * n + t] = (r <= c) ? ri[t] : 0.0;
    }
    if (threadIdx.x == 0) {
        double mn = 1e300, mx = 0.0;
        for (int r = 0; r < n; ++r) {
            mn = fmin(mn, fabs(a[r + n * r]));
            mx = fmax(mx, fabs(a[r + n * r]));
        }
        if (ratio) ratio[s] = mn / mx;
        if (bad) atomicCAS(err, 0, (int)SFM_ERR_BREAKDOWN);
    }
}

// C = A * B for small n x n blocks in shared memory (column-major)
__device__ void sm_gemm(const double* A, const double* B, double* C, int n, bool ta, bool tb) {
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int r = t % n, c = t / n;
        double v = 0.0;
        for (int l = 0; l < n; ++l) {
            const double a = ta ? A[l + n * r] : A[r + n * l];
            const double b = tb ? B[c + n * l] : B[l + n * c];
            v += a * b;
        }
        C[t] = v;
    }
}

// In-place inverse of a general n x n matrix (column-major) by Gauss-Jordan
// with partial pivoting; W is n*n scratch.  Returns false if singular.
__device__ bool sm_inverse(double* A, double* W, int n, int* piv) {
    __shared__ int ok;
    if (threadIdx.x == 0) ok = 1;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) W[t] = ((t % n) == (t / n)) ? 1.0 : 0.0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            int p = j;
            double best = fabs(A[j + n * j]);
            for (int r = j + 1; r < n; ++r)
                if (fabs(A[r + n * j]) > best) { best = fabs(A[r + n * j]); p = r; }
            piv[0] = p;
            if (best == 0.0) ok = 0;
        }
        __syncthreads();
        const int p = piv[0];
        if (p != j) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                double t1 = A[j + n * c]; A[j + n * c] = A[p + n * c]; A[p + n * c] = t1;
                double t2 = W[j + n * c]; W[j + n * c] = W[p + n * c]; W[p + n * c] = t2;
            }
        }
        __syncthreads();
        const double d = A[j + n * j];
        __syncthreads();
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            A[j + n * c] /= d;
            W[j + n * c] /= d;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int r = t % n, c = t / n;
            if (r != j) {
                const double f = A[r + n * j];
                // A[r, j] itself is cleared by the c == j term below
                if (c != j) A[r + n * c] -= f * A[j + n * c];
                W[r + n * c] -= f * W[j + n * c];
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x)
            if (r != j) A[r + n * j] = 0.0;
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = W[t];
    __syncthreads();
    return ok != 0;
}

// S-fraction transform (Eq. 13) of one subdomain per block:
//   G_1 = R_1^T, Gammahat_j = G_j G_j^T, Gamma_j = G_j^{-T} alpha_j G_j^{-1} - Gamma_{j-1},
//   G_{j+1} = -(G_j^T Gamma_j)^{-1} C_{j+1}^T.
// alpha: k blocks, C: k-1 blocks (block (j+1, j) of T_L), R1: b x b; all
// column-major b x b.  Outputs Gamma, Gammahat (k blocks each, symmetrised)
// and Ginv (k blocks: G_j^{-1}).  err = SFM_ERR_NOT_SPD when a diagonal of
// Gamma_j, j < k, is not positive (a cheap necessary check).  Work space 5 b*b:
// dynamic shared memory, or the block's slice of ws for wide blocks.
__global__ void gamma_kernel(const double* alpha, const double* C, const double* R1, int b, int k,
                             double* Gam, double* Gh, double* Ginv, int* err, double* ws) {
    // alpha: [S][k] blocks; C: level-major [k-1][S] blocks; R1: [S]
    extern __shared__ double sm_dyn[];
    const int bb = b * b;
    double* sm = ws ? ws + (long long)blockIdx.x * 5 * bb : sm_dyn;
    double* G = sm;
    double* Gi = sm + bb;
    double* prev = sm + 2 * bb;
    double* T1 = sm + 3 * bb;
    double* T2 = sm + 4 * bb;
    __shared__ int piv[1];
    const long long s = blockIdx.x;
    const double* al = alpha + s * k * bb;
    const long long S_ = gridDim.x;
    for (int t = threadIdx.x; t < bb; t += blockDim.x) {
        const int r = t % b, c = t / b;
        G[t] = R1[s * bb + c + b * r];   // R1^T
        prev[t] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        // Gammahat_j = G G^T
        sm_gemm(G, G, T1, b, false, true);
        __syncthreads();
        for (int t = threadIdx.x; t < bb; t += blockDim.x) {
            const int r = t % b, c = t / b;
            Gh[(s * k + j) * bb + t] = 0.5 * (T1[t] + T1[c + b * r]);
        }
        // Gi = G^{-1}
        for (int t = threadIdx.x; t < bb; t += blockDim.x) Gi[t] = G[t];
        __syncthreads();
        if (!sm_inverse(Gi, T2, b, piv)) {
            if (threadIdx.x == 0) atomicCAS(err, 0, (int)SFM_ERR_BREAKDOWN);
            return;
        }
        for (int t = threadIdx.x; t < bb; t += blockDim.x) Ginv[(s * k + j) * bb + t] = Gi[t];
        // Gamma_j = Gi^T alpha_j Gi - prev
        for (int t = threadIdx.x; t < bb; t += blockDim.x) {
            const int r = t % b, c = t / b;
            T2[t] = 0.5 * (al[j * bb + t] + al[j * bb + c + b * r]);
        }
        __syncthreads();
        sm_gemm(Gi, T2, T1, b, true, false);   // Gi^T alpha
        __syncthreads();
        sm_gemm(T1, Gi, T2, b, false, false);  // (Gi^T alpha) Gi
        __syncthreads();
        for (int t = threadIdx.x; t < bb; t += blockDim.x) {
            const int r = t % b, c = t / b;
            T1[t] = 0.5 * (T2[t] + T2[c + b * r]) - prev[t];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < bb; t += blockDim.x) {
            const int r = t % b, c = t / b;
            const double v = 0.5 * (T1[t] + T1[c + b * r]);
            prev[t] = v;
            Gam[(s * k + j) * bb + t] = v;
        }
        __syncthreads();
        if (j < k - 1 && threadIdx.x == 0) {
            for (int r = 0; r < b; ++r)
                if (!(prev[r + b * r] > 0.0)) { atomicCAS(err, 0, (int)SFM_ERR_NOT_SPD); break; }
        }
        if (j == k - 1) break;
        // G_{j+1} = -(G^T Gamma_j)^{-1} C_{j+1}^T
        sm_gemm(G, prev, T1, b, true, false);   // G^T Gamma_j
        __syncthreads();
        if (!sm_inverse(T1, T2, b, piv)) {
            if (threadIdx.x == 0) atomicCAS(err, 0, (int)SFM_ERR_BREAKDOWN);
            return;
        }
        for (int t = threadIdx.x; t < bb; t += blockDim.x) T2[t] = C[((long long)j * S_ + s) * bb + t];
        __syncthreads();
        sm_gemm(T1, T2, G, b, false, true);      // (G^T Gamma)^{-1} C^T
        __syncthreads();
        for (int t = threadIdx.x; t < bb; t += blockDim.x) G[t] = -G[t];
        __syncthreads();
    }
}

// Gather rows: y[s][c] = sum over the pair's nodes w_i * V[s][c][node_i] / sqrt(m[s][node_i])
// for one (point, subdomain) pair per block; V column-major N x ncol.
__global__ void gather_project_kernel(const double* V, const double* mass, int N, int ncol,
                                      const int* pair_sub_local, const int* node_ptr,
                                      const int* nodes, const double* wts, double* Y) {
    const int pr = blockIdx.x;
    const int s = pair_sub_local[pr];
    const double* Vs = V + (long long)s * N * ncol;
    const double* m = mass + (long long)s * N;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double acc = 0.0;
        for (int e = node_ptr[pr]; e < node_ptr[pr + 1]; ++e) {
            const int n = nodes[e];
            acc += wts[e] * Vs[(long long)c * N + n] / sqrt(m[n]);
        }
        Y[(long long)pr * ncol + c] = acc;
    }
}

// rows[pr][j][:] = Ginv_j^T z_j for z = Qh^T y (z given), one pair per block
__global__ void finish_project_kernel(const double* Z, const double* Ginv, int b, int k,
                                      const int* pair_sub_local, double* rows) {
    const int pr = blockIdx.x;
    const int s = pair_sub_local[pr];
    const int bb = b * b;
    for (int t = threadIdx.x; t < k * b; t += blockDim.x) {
        const int j = t / b, i = t % b;
        const double* Gi = Ginv + ((long long)s * k + j) * bb;   // column-major
        double acc = 0.0;
        for (int l = 0; l < b; ++l) acc += Gi[l + b * i] * Z[(long long)pr * k * b + j * b + l];
        rows[(long long)pr * k * b + t] = acc;
    }
}

}  // namespace bld

// Positive semi-definiteness of the finished S-fraction blocks (FP64
// masters, per subdomain Gamma_1..k then Gammahat_1..k, b x b).  One block
// of threads per (subdomain, block).  A Cholesky test in shared memory
// leaves a block that factors untouched; a block that meets a non-positive
// pivot (deep levels whose smallest eigenvalues sit at the FP64 rounding
// level, where rounding makes some slightly negative) is replaced by its
// projection on the positive semi-definite cone, V max(Lambda, 0) V^T, from
// a cyclic Jacobi eigen-decomposition; such blocks are counted.  A shift
// would be wrong here: it gives a singular inverse-mass direction a finite
// mass, and with the large stiffness paired with it a spurious fast mode.
// Blocks up to 64 wide work in shared memory (A and V, 64 rows of 65);
// wider ones in the block's slice of the global work space ws (2 b(b+1)
// numbers a block, rows of b + 1).
constexpr int PSD_NARROW_LD = 65;
constexpr size_t PSD_SMEM = 2 * 64 * PSD_NARROW_LD * sizeof(double);
__global__ void __launch_bounds__(256) psd_project_kernel(double* coef, const long long* coef_off,
                                                          const int* sub_b, const int* sub_k,
                                                          int* nproj, double* ws, int bmax) {
    extern __shared__ double psd_smem[];
    const int REG_LD = ws ? bmax + 1 : PSD_NARROW_LD;
    double* A = ws ? ws + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2LL * bmax * REG_LD : psd_smem;
    double* V = A + (ws ? bmax : 64) * REG_LD;
    __shared__ double s_cs[2];
    __shared__ int s_ok;
    const int s = blockIdx.y, blk = blockIdx.x;
    const int b = sub_b[s], k = sub_k[s];
    if (blk >= 2 * k) return;
    double* m = coef + coef_off[s] + (long long)blk * b * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) A[(e / b) * REG_LD + e % b] = m[e];
    // Cholesky test
    bool ok = true;
    for (int c = 0; c < b; ++c) {
        __syncthreads();
        const double d = A[c * REG_LD + c];
        if (!(d > 0.0)) { ok = false; break; }
        const double l = sqrt(d);
        __syncthreads();
        if (threadIdx.x == 0) A[c * REG_LD + c] = l;
        for (int i = c + 1 + threadIdx.x; i < b; i += blockDim.x) A[i * REG_LD + c] /= l;
        __syncthreads();
        const int n = b - c - 1;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = c + 1 + t / n, jj = c + 1 + t % n;
            if (jj <= i) A[i * REG_LD + jj] -= A[i * REG_LD + c] * A[jj * REG_LD + c];
        }
    }
    __syncthreads();
    if (ok) return;
    // cyclic Jacobi on the symmetrised block
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        A[i * REG_LD + j] = 0.5 * (m[i * b + j] + m[j * b + i]);
        V[i * REG_LD + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (threadIdx.x == 0) {
            double off = 0.0, dia = 0.0;
            for (int i = 0; i < b; ++i)
                for (int j = 0; j < b; ++j)
                    (i == j ? dia : off) += A[i * REG_LD + j] * A[i * REG_LD + j];
            s_ok = (off <= 1e-30 * dia) ? 1 : 0;
        }
        __syncthreads();
        if (s_ok) break;
        for (int pp = 0; pp < b - 1; ++pp) {
            for (int qq = pp + 1; qq < b; ++qq) {
                if (threadIdx.x == 0) {
                    const double apq = A[pp * REG_LD + qq];
                    double c = 1.0, sn = 0.0;
                    if (apq != 0.0) {
                        const double tau = (A[qq * REG_LD + qq] - A[pp * REG_LD + pp]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                    }
                    s_cs[0] = c;
                    s_cs[1] = sn;
                }
                __syncthreads();
                const double c = s_cs[0], sn = s_cs[1];
                if (sn != 0.0) {
                    // A <- J^T A J on rows and columns pp, qq; V <- V J
                    for (int i = threadIdx.x; i < b; i += blockDim.x) {
                        const double aip = A[i * REG_LD + pp], aiq = A[i * REG_LD + qq];
                        A[i * REG_LD + pp] = c * aip - sn * aiq;
                        A[i * REG_LD + qq] = sn * aip + c * aiq;
                        const double vip = V[i * REG_LD + pp], viq = V[i * REG_LD + qq];
                        V[i * REG_LD + pp] = c * vip - sn * viq;
                        V[i * REG_LD + qq] = sn * vip + c * viq;
                    }
                    __syncthreads();
                    for (int j = threadIdx.x; j < b; j += blockDim.x) {
                        const double apj = A[pp * REG_LD + j], aqj = A[qq * REG_LD + j];
                        A[pp * REG_LD + j] = c * apj - sn * aqj;
                        A[qq * REG_LD + j] = sn * apj + c * aqj;
                    }
                }
                __syncthreads();
            }
        }
    }
    // m = V max(diag A, 0) V^T
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        double acc = 0.0;
        for (int t = 0; t < b; ++t) {
            const double lam = A[t * REG_LD + t];
            if (lam > 0.0) acc += V[i * REG_LD + t] * lam * V[j * REG_LD + t];
        }
        m[e] = acc;
    }
    if (threadIdx.x == 0) atomicAdd(nproj, 1);
}

}  // namespace sfm
