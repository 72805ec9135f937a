// FP64 offline ROM builder on the GPU (Algorithm 1 stage 1, steps 1.1-1.4):
// fine operator, face basis, shifted block Krylov subspace (Eqs. 6-7 with a
// single repeated shift and F as the first block), Galerkin ROM (Eq. 5),
// block Lanczos (Eq. 8) and the S-fraction transform (Eq. 13), then the
// projection of point sources and receivers (Eq. 16).
//
// Subdomains are processed in classes of equal shape (cells per axis, face
// mode counts, k), each class as one batch: the shifted solves are a
// Jacobi-preconditioned CG over every (subdomain, column) pair at once, the
// Gram-Schmidt, Galerkin and Lanczos products are strided-batched cuBLAS
// DGEMMs, and the small b x b factorisations run one block per matrix.
#include "sfm_internal.h"
#include "builder_kernels.cuh"

#include <cublas_v2.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <tuple>

namespace {

using sfm::bld::ColSpec;

struct BClass {
    int nxl = 0, nyl = 0, nzl = 0, b = 0, k = 0, N = 0;
    int mf[6] = {0, 0, 0, 0, 0, 0};
    std::vector<int> subs;
    double* mass = nullptr;    // S x N
    double* V = nullptr;       // S x (N x bk), column-major
    double* Qh = nullptr;      // S x (bk x bk)
    double* Ginv = nullptr;    // S x k x (b x b)
    int3* origin = nullptr;
};

struct BuildState {
    int gnx = 0, gny = 0, gnz = 0;
    double h = 0.0;
    double* d_c = nullptr;
    double* d_gmass = nullptr;        // global lumped mass, (gnx+1)(gny+1)(gnz+1)
    std::vector<int> xc, yc, zc;
    std::vector<BClass> classes;
    std::vector<int> sub_class, sub_pos;
    std::vector<int> m_sub, k_sub;
    double sigma = 0.0;
    bool built = false;
    cublasHandle_t blas = nullptr;
};

template <typename P>
void dfree(P*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_classes(BuildState* b) {
    for (auto& c : b->classes) {
        dfree(c.mass); dfree(c.V); dfree(c.Qh); dfree(c.Ginv); dfree(c.origin);
    }
    b->classes.clear();
    b->built = false;
}

BuildState* bstate(sfm_handle* h) { return reinterpret_cast<BuildState*>(h->build); }

int bfail(sfm_handle* h, int code, const std::string& msg) {
    h->err = msg;
    return code;
}

#define BCK(h, call)                                                                  \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess)                                                       \
            return bfail((h), e__ == cudaErrorMemoryAllocation ? SFM_ERR_NOMEM : SFM_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e__));        \
    } while (0)

#define BLK(h, call)                                                                  \
    do {                                                                              \
        cublasStatus_t s__ = (call);                                                  \
        if (s__ != CUBLAS_STATUS_SUCCESS)                                             \
            return bfail((h), SFM_ERR_CUDA, std::string(#call) + ": cublas status " + \
                                                std::to_string((int)s__));            \
    } while (0)

// Frees the device temporaries it names when it leaves scope, so that an
// error return does not leak them (those already freed are null).
template <typename... P>
struct DevGuard {
    std::tuple<P*&...> ptrs;
    explicit DevGuard(P*&... p) : ptrs(p...) {}
    ~DevGuard() { std::apply([](auto&... q) { (dfree(q), ...); }, ptrs); }
    DevGuard(const DevGuard&) = delete;
    DevGuard& operator=(const DevGuard&) = delete;
};

template <typename P>
cudaError_t dmalloc(P*& p, size_t count) {
    dfree(p);
    return cudaMalloc((void**)&p, (count ? count : 1) * sizeof(P));
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1LL, std::min(g, 65535LL * 8));
}

// Modes of one face in the order of ascending p^2 + q^2, then q, then p.
std::vector<std::pair<int, int>> face_modes(int ns, int nt, int m) {
    std::vector<std::tuple<int, int, int, int>> all;
    for (int p = 0; p < ns; ++p)
        for (int q = 0; q < nt; ++q) all.emplace_back(p * p + q * q, q, p, 0);
    std::sort(all.begin(), all.end());
    std::vector<std::pair<int, int>> out;
    for (int i = 0; i < m && i < (int)all.size(); ++i)
        out.emplace_back(std::get<2>(all[i]), std::get<1>(all[i]));
    return out;
}

struct Gemm {
    cublasHandle_t h;
    // C[s] = alpha op(A[s]) op(B[s]) + beta C[s]; column-major
    cublasStatus_t operator()(bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
                              int lda, long long sA, const double* B, int ldb, long long sB,
                              double beta, double* C, int ldc, long long sC, int batch) const {
        return cublasDgemmStridedBatched(h, ta ? CUBLAS_OP_T : CUBLAS_OP_N,
                                         tb ? CUBLAS_OP_T : CUBLAS_OP_N, m, n, k, &alpha, A, lda,
                                         sA, B, ldb, sB, &beta, C, ldc, sC, batch);
    }
};

}  // namespace

namespace sfm {
void free_build(sfm_handle* h) {
    BuildState* b = bstate(h);
    if (!b) return;
    free_classes(b);
    dfree(b->d_c);
    dfree(b->d_gmass);
    if (b->blas) cublasDestroy(b->blas);
    delete b;
    h->build = nullptr;
}
int set_topology_internal(sfm_handle* h, int nsub, const int* k_sub, const int* m_face,
                          const int* nbr);
int set_coeffs_device(sfm_handle* h, const double* d_coeffs);
}  // namespace sfm

// Largest dynamic shared memory the builder's one-block-per-matrix kernels
// take; wider blocks work in global memory.
constexpr size_t kBuilderSmem = 200 * 1024;

// Orthonormalise a batch of N x n blocks in place by Cholesky QR done twice:
// X = Q R with R = R2 R1.  Rout (S x n x n) receives R when not NULL.
static int cholqr2(sfm_handle* h, const Gemm& gemm, double* X, long long sX, int N, int n, int S,
                   double* tmp, double* Gm, double* R1, double* R1i, double* R2, double* R2i,
                   double* Rout, int* d_err, double* d_ratio, double* min_ratio) {
    cudaStream_t st = h->stream;
    const long long nn = (long long)n * n;
    // work space of the factorisation: shared memory, or global for wide blocks
    size_t smem = 2 * nn * sizeof(double);
    double* ws = nullptr;
    DevGuard guard_ws(ws);
    if (smem > kBuilderSmem) {
        BCK(h, dmalloc(ws, (size_t)S * 2 * nn));
        smem = 0;
    } else {
        BCK(h, cudaFuncSetAttribute(sfm::bld::chol_rinv_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    for (int pass = 0; pass < 2; ++pass) {
        double* R = pass ? R2 : R1;
        double* Ri = pass ? R2i : R1i;
        BLK(h, gemm(true, false, n, n, N, 1.0, X, N, sX, X, N, sX, 0.0, Gm, n, nn, S));
        sfm::bld::chol_rinv_kernel<<<S, 128, smem, st>>>(Gm, R, Ri, n, d_err,
                                                          pass == 0 ? d_ratio : nullptr, ws);
        BCK(h, cudaGetLastError());
        BLK(h, gemm(false, false, N, n, n, 1.0, X, N, sX, Ri, n, nn, 0.0, tmp, N, (long long)N * n, S));
        BCK(h, cudaMemcpy2DAsync(X, sX * sizeof(double), tmp, (size_t)N * n * sizeof(double),
                                 (size_t)N * n * sizeof(double), S, cudaMemcpyDeviceToDevice, st));
    }
    if (Rout) BLK(h, gemm(false, false, n, n, n, 1.0, R2, n, nn, R1, n, nn, 0.0, Rout, n, nn, S));
    if (min_ratio) {
        std::vector<double> r(S);
        BCK(h, cudaMemcpyAsync(r.data(), d_ratio, S * sizeof(double), cudaMemcpyDeviceToHost, st));
        BCK(h, cudaStreamSynchronize(st));
        for (double v : r) *min_ratio = std::min(*min_ratio, v);
    }
    return SFM_OK;
}

extern "C" int sfm_set_model(sfm_handle* h, int nx, int ny, int nz, double hgrid, const double* c,
                             int ncx, const int* xcuts, int ncy, const int* ycuts, int ncz,
                             const int* zcuts) {
    if (!h) return SFM_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || !(hgrid > 0) || !c || ncx < 1 || ncy < 1 || ncz < 1 ||
        !xcuts || !ycuts || !zcuts)
        return bfail(h, SFM_ERR_ARG, "sfm_set_model: bad arguments");
    auto check_cuts = [](int n, int nc, const int* cuts) {
        if (cuts[0] != 0 || cuts[nc] != n) return false;
        for (int i = 0; i < nc; ++i)
            if (cuts[i + 1] - cuts[i] < 2) return false;   // an open face needs >= 2 cells
        return true;
    };
    if (!check_cuts(nx, ncx, xcuts) || !check_cuts(ny, ncy, ycuts) || !check_cuts(nz, ncz, zcuts))
        return bfail(h, SFM_ERR_ARG, "sfm_set_model: cuts must run 0..n with >= 2 cells each");
    const size_t ncell = (size_t)nx * ny * nz;
    for (size_t i = 0; i < ncell; ++i)
        if (!(c[i] > 0.0) || !std::isfinite(c[i]))
            return bfail(h, SFM_ERR_ARG, "sfm_set_model: velocities must be positive and finite");
    BCK(h, cudaSetDevice(h->device));
    if (!bstate(h)) {
        h->build = new BuildState();
        if (cublasCreate(&bstate(h)->blas) != CUBLAS_STATUS_SUCCESS)
            return bfail(h, SFM_ERR_CUDA, "cublasCreate failed");
    }
    BuildState* b = bstate(h);
    free_classes(b);
    b->gnx = nx; b->gny = ny; b->gnz = nz; b->h = hgrid;
    b->xc.assign(xcuts, xcuts + ncx + 1);
    b->yc.assign(ycuts, ycuts + ncy + 1);
    b->zc.assign(zcuts, zcuts + ncz + 1);
    BCK(h, dmalloc(b->d_c, ncell));
    BCK(h, cudaMemcpyAsync(b->d_c, c, ncell * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // global lumped mass (used for the shares of shared nodes in step 1.4)
    const size_t ng = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    BCK(h, dmalloc(b->d_gmass, ng));
    int3* o = nullptr;
    BCK(h, dmalloc(o, 1));
    const int3 z0 = make_int3(0, 0, 0);
    BCK(h, cudaMemcpyAsync(o, &z0, sizeof(int3), cudaMemcpyHostToDevice, h->stream));
    sfm::bld::mass_kernel<<<grid_for((long long)ng), 256, 0, h->stream>>>(b->d_c, nx, ny, o, 1, nx, ny,
                                                                          nz, hgrid, b->d_gmass);
    BCK(h, cudaGetLastError());
    BCK(h, cudaStreamSynchronize(h->stream));
    dfree(o);
    return SFM_OK;
}

// The exact build (Algorithm 1 steps 1.1-1.3).  only: when not NULL, just the
// subdomains with only[s] != 0 are built (the others keep the coefficients
// of d_preset, a full coefficient array on the device, and have no Krylov
// basis for the projections of step 1.4).
static int build_impl(sfm_handle* h, const int* m_sub, const int* k_sub, double sigma, double cg_tol,
                      sfm_build_report* rep, const std::vector<char>* only, const double* d_preset,
                      const double* shifts = nullptr) {
    if (!h) return SFM_ERR_ARG;
    BuildState* B = bstate(h);
    if (!B || !B->d_c) return bfail(h, SFM_ERR_STATE, "sfm_build_roms: no model");
    if (!m_sub || !k_sub || !(sigma > 0.0))
        return bfail(h, SFM_ERR_ARG, "sfm_build_roms: bad arguments");
    if (!(cg_tol > 0.0)) cg_tol = 1e-14;
    BCK(h, cudaSetDevice(h->device));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = h->stream;
    cublasSetStream(B->blas, st);
    cublasSetPointerMode(B->blas, CUBLAS_POINTER_MODE_HOST);
    const Gemm gemm{B->blas};
    const int ncx = (int)B->xc.size() - 1, ncy = (int)B->yc.size() - 1, ncz = (int)B->zc.size() - 1;
    const int nsub = ncx * ncy * ncz;
    free_classes(B);
    B->m_sub.assign(m_sub, m_sub + nsub);
    B->k_sub.assign(k_sub, k_sub + nsub);
    B->sigma = sigma;

    // topology: neighbours across the 6 faces, modes per face
    std::vector<int> nbr(6 * nsub, -1), mface(6 * nsub, 0);
    for (int s = 0; s < nsub; ++s) {
        if (k_sub[s] < 1 || m_sub[s] < 1) return bfail(h, SFM_ERR_ARG, "sfm_build_roms: m, k >= 1");
        const int pos[3] = {s % ncx, (s / ncx) % ncy, s / (ncx * ncy)};
        const int lim[3] = {ncx, ncy, ncz};
        for (int f = 0; f < 6; ++f) {
            int q[3] = {pos[0], pos[1], pos[2]};
            q[f / 2] += (f & 1) ? 1 : -1;
            if (q[f / 2] >= 0 && q[f / 2] < lim[f / 2]) nbr[s * 6 + f] = q[0] + ncx * (q[1] + ncy * q[2]);
        }
    }
    for (int s = 0; s < nsub; ++s)
        for (int f = 0; f < 6; ++f) {
            const int t = nbr[s * 6 + f];
            mface[s * 6 + f] = (t < 0) ? m_sub[s] : std::min(m_sub[s], m_sub[t]);
        }
    // classes of equal shape
    std::map<std::vector<int>, int> cls;
    B->sub_class.assign(nsub, 0);
    B->sub_pos.assign(nsub, 0);
    for (int s = 0; s < nsub; ++s) {
        if (only && !(*only)[s]) {
            B->sub_class[s] = -1;
            continue;
        }
        const int ix = s % ncx, iy = (s / ncx) % ncy, iz = s / (ncx * ncy);
        std::vector<int> key = {B->xc[ix + 1] - B->xc[ix], B->yc[iy + 1] - B->yc[iy],
                                B->zc[iz + 1] - B->zc[iz], k_sub[s]};
        for (int f = 0; f < 6; ++f) key.push_back(mface[s * 6 + f]);
        auto it = cls.find(key);
        int ci;
        if (it == cls.end()) {
            ci = (int)B->classes.size();
            cls[key] = ci;
            BClass c;
            c.nxl = key[0]; c.nyl = key[1]; c.nzl = key[2]; c.k = key[3];
            c.b = 0;
            for (int f = 0; f < 6; ++f) { c.mf[f] = key[4 + f]; c.b += c.mf[f]; }
            c.N = (c.nxl + 1) * (c.nyl + 1) * (c.nzl + 1);
            B->classes.push_back(c);
        } else {
            ci = it->second;
        }
        B->sub_class[s] = ci;
        B->sub_pos[s] = (int)B->classes[ci].subs.size();
        B->classes[ci].subs.push_back(s);
    }
    for (auto& c : B->classes) {
        const int ncell[3] = {c.nxl, c.nyl, c.nzl};
        for (int f = 0; f < 6; ++f) {
            const int a = f / 2, u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2;
            if (c.mf[f] > (ncell[u] - 1) * (ncell[v] - 1))
                return bfail(h, SFM_ERR_ARG, "sfm_build_roms: more modes than open-face nodes");
        }
        if (c.b > sfm::BMAX_WIDE)
            return bfail(h, SFM_ERR_ARG, "sfm_build_roms: block width b above " + std::to_string(sfm::BMAX_WIDE));
    }
    int rc = sfm::set_topology_internal(h, nsub, k_sub, mface.data(), nbr.data());
    if (rc != SFM_OK) return rc;

    // device coefficient array in the stepping layout
    double* d_coef = nullptr;
    BCK(h, dmalloc(d_coef, (size_t)h->ncoef));
    if (d_preset)
        BCK(h, cudaMemcpyAsync(d_coef, d_preset, (size_t)h->ncoef * sizeof(double), cudaMemcpyDeviceToDevice, st));

    int* d_err = nullptr;
    double* d_ratio = nullptr;
    DevGuard guard_top(d_coef, d_err, d_ratio);
    BCK(h, dmalloc(d_err, 1));
    BCK(h, cudaMemsetAsync(d_err, 0, sizeof(int), st));
    int cg_iters_max = 0;
    double cg_res_max = 0.0, min_ratio = 1.0;

    for (auto& c : B->classes) {
        const int S = (int)c.subs.size(), N = c.N, b = c.b, k = c.k, n = b * k;
        const long long bb = (long long)b * b;
        // origins
        std::vector<int3> org(S);
        for (int i = 0; i < S; ++i) {
            const int s = c.subs[i];
            org[i] = make_int3(B->xc[s % ncx], B->yc[(s / ncx) % ncy], B->zc[s / (ncx * ncy)]);
        }
        BCK(h, dmalloc(c.origin, S));
        BCK(h, cudaMemcpyAsync(c.origin, org.data(), S * sizeof(int3), cudaMemcpyHostToDevice, st));
        BCK(h, dmalloc(c.mass, (size_t)S * N));
        sfm::bld::mass_kernel<<<grid_for((long long)S * N), 256, 0, st>>>(
            B->d_c, B->gnx, B->gny, c.origin, S, c.nxl, c.nyl, c.nzl, B->h, c.mass);
        BCK(h, cudaGetLastError());
        // face basis B (shared by the class)
        std::vector<ColSpec> cs;
        const int ncell[3] = {c.nxl, c.nyl, c.nzl};
        for (int f = 0; f < 6; ++f) {
            const int a = f / 2, u = (a == 0) ? 1 : 0, v = (a == 2) ? 1 : 2;
            for (auto pq : face_modes(ncell[u] - 1, ncell[v] - 1, c.mf[f]))
                cs.push_back({f, pq.first, pq.second, 0});
        }
        ColSpec* d_cs = nullptr;
        double* Bm = nullptr;
        DevGuard guard_basis(d_cs, Bm);
        BCK(h, dmalloc(d_cs, cs.size()));
        BCK(h, cudaMemcpyAsync(d_cs, cs.data(), cs.size() * sizeof(ColSpec), cudaMemcpyHostToDevice, st));
        BCK(h, dmalloc(Bm, (size_t)N * b));
        sfm::bld::basis_kernel<<<grid_for((long long)N * b), 256, 0, st>>>(d_cs, b, c.nxl, c.nyl,
                                                                            c.nzl, B->h, Bm);
        BCK(h, cudaGetLastError());
        // work buffers
        const long long sV = (long long)N * n;
        double *tmp = nullptr, *Gm = nullptr, *R1 = nullptr, *R1i = nullptr, *R2 = nullptr,
               *R2i = nullptr, *Rr = nullptr;
        DevGuard guard_work(tmp, Gm, R1, R1i, R2, R2i, Rr);
        BCK(h, dmalloc(c.V, (size_t)S * sV));
        BCK(h, dmalloc(tmp, (size_t)S * N * b));
        BCK(h, dmalloc(Gm, (size_t)S * n * b));
        BCK(h, dmalloc(R1, (size_t)S * bb));
        BCK(h, dmalloc(R1i, (size_t)S * bb));
        BCK(h, dmalloc(R2, (size_t)S * bb));
        BCK(h, dmalloc(R2i, (size_t)S * bb));
        BCK(h, dmalloc(Rr, (size_t)S * bb));
        BCK(h, dmalloc(d_ratio, (size_t)S));
        // F = M^{-1/2} B -> block 0, then Q_1
        sfm::bld::scale_kernel<<<grid_for((long long)S * N * b), 256, 0, st>>>(Bm, 0, c.mass, c.V, sV,
                                                                               N, b, S, 1);
        BCK(h, cudaGetLastError());
        rc = cholqr2(h, gemm, c.V, sV, N, b, S, tmp, Gm, R1, R1i, R2, R2i, nullptr, d_err, d_ratio,
                     nullptr);
        if (rc) return rc;
        // shifted block Krylov with CG solves of (K + sigma M)
        double *Xc = nullptr, *Rc = nullptr, *Zc = nullptr, *Pc = nullptr, *Qc = nullptr,
               *rhs = nullptr, *rz = nullptr, *rz2 = nullptr, *pq = nullptr, *rr = nullptr,
               *rr0 = nullptr;
        DevGuard guard_cg(Xc, Rc, Zc, Pc, Qc, rhs, rz, rz2, pq, rr, rr0);
        const size_t ncolv = (size_t)S * b;
        if (k > 1) {
            for (double** p : {&Xc, &Rc, &Zc, &Pc, &Qc, &rhs}) BCK(h, dmalloc(*p, ncolv * N));
            for (double** p : {&rz, &rz2, &pq, &rr, &rr0}) BCK(h, dmalloc(*p, ncolv));
        }
        std::vector<double> h_rr(ncolv), h_rr0(ncolv);
        for (int j = 1; j < k; ++j) {
            double* Qj = c.V + (long long)(j - 1) * N * b;
            double* Wj = c.V + (long long)j * N * b;
            // block j+1 = (L + sigma_j)^{-1} block j: one shift repeated, or
            // the j-th of distinct shifts (Eq. 6)
            const double sig = shifts ? shifts[j - 1] : sigma;
            // rhs = M^{1/2} Q_j
            sfm::bld::scale_kernel<<<grid_for((long long)ncolv * N), 256, 0, st>>>(Qj, sV, c.mass, rhs,
                                                                                   (long long)N * b, N,
                                                                                   b, S, 0);
            sfm::bld::cg_init_kernel<<<(int)ncolv, 256, 0, st>>>(rhs, Xc, Rc, Zc, Pc, c.mass, c.nxl, c.nyl,
                                                                 c.nzl, B->h, sig, b, rz, rr0);
            BCK(h, cudaGetLastError());
            BCK(h, cudaMemcpyAsync(h_rr0.data(), rr0, ncolv * sizeof(double), cudaMemcpyDeviceToHost, st));
            int it = 0;
            double worst = 0.0;
            const int max_it = 20000;
            for (it = 1; it <= max_it; ++it) {
                sfm::bld::op_kernel<<<(int)ncolv, 256, 0, st>>>(Pc, Qc, c.mass, c.nxl, c.nyl, c.nzl,
                                                                B->h, sig, b, 0, pq);
                sfm::bld::cg_update_kernel<<<(int)ncolv, 256, 0, st>>>(Xc, Rc, Zc, Pc, Qc, c.mass, c.nxl,
                                                                       c.nyl, c.nzl, B->h, sig, b,
                                                                       rz, pq, rz2, rr);
                sfm::bld::cg_dir_kernel<<<(int)ncolv, 256, 0, st>>>(Pc, Zc, N, rz, rz2);
                if (it % 8 == 0) {
                    BCK(h, cudaGetLastError());
                    BCK(h, cudaMemcpyAsync(h_rr.data(), rr, ncolv * sizeof(double),
                                           cudaMemcpyDeviceToHost, st));
                    BCK(h, cudaStreamSynchronize(st));
                    worst = 0.0;
                    for (size_t i = 0; i < ncolv; ++i)
                        if (h_rr0[i] > 0) worst = std::max(worst, std::sqrt(h_rr[i] / h_rr0[i]));
                    if (worst < cg_tol) break;
                }
            }
            if (it > max_it) return bfail(h, SFM_ERR_BREAKDOWN, "sfm_build_roms: CG did not converge");
            cg_iters_max = std::max(cg_iters_max, it);
            cg_res_max = std::max(cg_res_max, worst);
            // W = M^{1/2} Y
            sfm::bld::scale_kernel<<<grid_for((long long)ncolv * N), 256, 0, st>>>(
                Xc, (long long)N * b, c.mass, Wj, sV, N, b, S, 0);
            BCK(h, cudaGetLastError());
            // block Gram-Schmidt against Q_1..Q_j, twice
            for (int pass = 0; pass < 2; ++pass) {
                BLK(h, gemm(true, false, j * b, b, N, 1.0, c.V, N, sV, Wj, N, sV, 0.0, Gm, j * b,
                            (long long)n * b, S));
                BLK(h, gemm(false, false, N, b, j * b, -1.0, c.V, N, sV, Gm, j * b, (long long)n * b, 1.0,
                            Wj, N, sV, S));
            }
            rc = cholqr2(h, gemm, Wj, sV, N, b, S, tmp, Gm, R1, R1i, R2, R2i, nullptr, d_err, d_ratio,
                         &min_ratio);
            if (rc) return rc;
        }
        for (double** p : {&Xc, &Rc, &Zc, &Pc, &rhs, &rz, &rz2, &pq, &rr, &rr0}) dfree(*p);
        // Galerkin ROM  L~ = V^T L V (column chunks), F~ = V^T F
        double *Lt = nullptr, *Ft = nullptr, *LVc = nullptr;
        DevGuard guard_rom(Lt, Ft, LVc);
        int chunk = std::min(n, 96);
        while (n % chunk) --chunk;                       // equal column chunks
        BCK(h, dmalloc(Lt, (size_t)S * n * n));
        BCK(h, dmalloc(Ft, (size_t)S * n * b));
        BCK(h, dmalloc(LVc, (size_t)S * N * chunk));
        double* Vcol = nullptr;
        DevGuard guard_vcol(Vcol);
        BCK(h, dmalloc(Vcol, (size_t)S * N * chunk));
        for (int c0 = 0; c0 < n; c0 += chunk) {
            const int w = std::min(chunk, n - c0);
            BCK(h, cudaMemcpy2DAsync(Vcol, (size_t)N * chunk * sizeof(double),
                                     c.V + (long long)c0 * N, sV * sizeof(double),
                                     (size_t)N * w * sizeof(double), S, cudaMemcpyDeviceToDevice, st));
            sfm::bld::op_kernel<<<S * w, 256, 0, st>>>(Vcol, LVc, c.mass, c.nxl, c.nyl, c.nzl, B->h, 0.0,
                                                        w, 1, nullptr);
            BCK(h, cudaGetLastError());
            BLK(h, gemm(true, false, n, w, N, 1.0, c.V, N, sV, LVc, N, (long long)N * chunk, 0.0,
                        Lt + (long long)c0 * n, n, (long long)n * n, S));
        }
        dfree(LVc);
        dfree(Vcol);
        // F = M^{-1/2} B again into tmp, F~ = V^T F
        sfm::bld::scale_kernel<<<grid_for((long long)S * N * b), 256, 0, st>>>(Bm, 0, c.mass, tmp,
                                                                               (long long)N * b, N, b, S, 1);
        BLK(h, gemm(true, false, n, b, N, 1.0, c.V, N, sV, tmp, N, (long long)N * b, 0.0, Ft, n,
                    (long long)n * b, S));
        dfree(Bm);
        dfree(d_cs);
        // block Lanczos on (L~, F~) with full reorthogonalisation
        double *al = nullptr, *Cm = nullptr, *Rl = nullptr, *Wl = nullptr, *tl = nullptr;
        DevGuard guard_lanczos(al, Cm, Rl, Wl, tl);
        BCK(h, dmalloc(c.Qh, (size_t)S * n * n));
        BCK(h, dmalloc(al, (size_t)S * k * bb));
        BCK(h, dmalloc(Cm, (size_t)S * std::max(1, k - 1) * bb));   // level-major [k-1][S]
        BCK(h, dmalloc(Rl, (size_t)S * bb));
        BCK(h, dmalloc(Wl, (size_t)S * n * b));
        BCK(h, dmalloc(tl, (size_t)S * n * b));
        const long long sQ = (long long)n * n;
        BCK(h, cudaMemcpy2DAsync(c.Qh, sQ * sizeof(double), Ft, (size_t)n * b * sizeof(double),
                                 (size_t)n * b * sizeof(double), S, cudaMemcpyDeviceToDevice, st));
        rc = cholqr2(h, gemm, c.Qh, sQ, n, b, S, tl, Gm, R1, R1i, R2, R2i, Rl, d_err, d_ratio, nullptr);
        if (rc) return rc;
        for (int j = 0; j < k; ++j) {
            double* Qj = c.Qh + (long long)j * n * b;
            BLK(h, gemm(false, false, n, b, n, 1.0, Lt, n, sQ, Qj, n, sQ, 0.0, Wl, n, (long long)n * b, S));
            BLK(h, gemm(true, false, b, b, n, 1.0, Qj, n, sQ, Wl, n, (long long)n * b, 0.0,
                        al + (long long)j * bb, b, (long long)k * bb, S));
            if (j == k - 1) break;
            BLK(h, gemm(false, false, n, b, b, -1.0, Qj, n, sQ, al + (long long)j * bb, b,
                        (long long)k * bb, 1.0, Wl, n, (long long)n * b, S));
            if (j > 0)
                BLK(h, gemm(false, true, n, b, b, -1.0, Qj - (long long)n * b, n, sQ,
                            Cm + (long long)(j - 1) * S * bb, b, bb, 1.0, Wl, n,
                            (long long)n * b, S));
            for (int pass = 0; pass < 2; ++pass) {
                BLK(h, gemm(true, false, (j + 1) * b, b, n, 1.0, c.Qh, n, sQ, Wl, n, (long long)n * b,
                            0.0, Gm, (j + 1) * b, (long long)n * b, S));
                BLK(h, gemm(false, false, n, b, (j + 1) * b, -1.0, c.Qh, n, sQ, Gm, (j + 1) * b,
                            (long long)n * b, 1.0, Wl, n, (long long)n * b, S));
            }
            rc = cholqr2(h, gemm, Wl, (long long)n * b, n, b, S, tl, Gm, R1, R1i, R2, R2i,
                         Cm + (long long)j * S * bb, d_err, d_ratio, nullptr);
            if (rc) return rc;
            // the orthonormalised block is Qh_{j+1}
            BCK(h, cudaMemcpy2DAsync(c.Qh + (long long)(j + 1) * n * b, sQ * sizeof(double), Wl,
                                     (size_t)n * b * sizeof(double), (size_t)n * b * sizeof(double), S,
                                     cudaMemcpyDeviceToDevice, st));
        }
        dfree(Lt); dfree(Ft); dfree(Wl); dfree(tl);
        // S-fraction transform
        double *Gam = nullptr, *Gh = nullptr;
        DevGuard guard_gamma(Gam, Gh);
        BCK(h, dmalloc(Gam, (size_t)S * k * bb));
        BCK(h, dmalloc(Gh, (size_t)S * k * bb));
        BCK(h, dmalloc(c.Ginv, (size_t)S * k * bb));
        size_t gsm = 5 * bb * sizeof(double);
        double* gws = nullptr;
        DevGuard guard_gws(gws);
        if (gsm > kBuilderSmem) {
            BCK(h, dmalloc(gws, (size_t)S * 5 * bb));   // wide blocks: global work space
            gsm = 0;
        } else {
            BCK(h, cudaFuncSetAttribute(sfm::bld::gamma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)gsm));
        }
        sfm::bld::gamma_kernel<<<S, 256, gsm, st>>>(al, Cm, Rl, b, k, Gam, Gh, c.Ginv, d_err, gws);
        BCK(h, cudaGetLastError());
        // scatter into the stepping layout: per subdomain Gamma_1..k then Gammahat_1..k
        for (int i = 0; i < S; ++i) {
            const int s = c.subs[i];
            BCK(h, cudaMemcpyAsync(d_coef + h->coef_off[s], Gam + (long long)i * k * bb,
                                   k * bb * sizeof(double), cudaMemcpyDeviceToDevice, st));
            BCK(h, cudaMemcpyAsync(d_coef + h->coef_off[s] + k * bb, Gh + (long long)i * k * bb,
                                   k * bb * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        BCK(h, cudaStreamSynchronize(st));
        for (double** p : {&al, &Cm, &Rl, &Gam, &Gh, &tmp, &Gm, &R1, &R1i, &R2, &R2i, &Rr, &Qc}) dfree(*p);
        dfree(d_ratio);
    }
    int herr = 0;
    BCK(h, cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCK(h, cudaStreamSynchronize(st));
    dfree(d_err);
    if (herr != 0) {
        dfree(d_coef);
        return bfail(h, herr, herr == SFM_ERR_NOT_SPD ? "sfm_build_roms: Gamma_j not positive definite"
                                                      : "sfm_build_roms: breakdown in a block factorisation");
    }
    // blocks that are semi-definite only up to FP64 rounding: projected on
    // the positive semi-definite cone (counted in the report)
    int nreg = 0;
    {
        int* d_nreg = nullptr;
        DevGuard guard_nreg(d_nreg);
        BCK(h, dmalloc(d_nreg, 1));
        BCK(h, cudaMemsetAsync(d_nreg, 0, sizeof(int), st));
        BCK(h, cudaFuncSetAttribute(sfm::psd_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sfm::PSD_SMEM));
        // blocks wider than 64: a global work space per launch block
        double* pws = nullptr;
        DevGuard guard_pws(pws);
        const size_t per_sub = (size_t)2 * h->kmax * 2 * h->bmax * (h->bmax + 1);   // doubles
        const int pchunk = (int)std::max<size_t>(1, std::min<size_t>(65535, (64u << 20) / per_sub));
        if (h->bmax > 64) BCK(h, dmalloc(pws, per_sub * pchunk));
        const int sstep = h->bmax > 64 ? pchunk : 65535;
        for (int s0 = 0; s0 < h->nsub; s0 += sstep) {
            const int ns = std::min(sstep, h->nsub - s0);
            sfm::psd_project_kernel<<<dim3(2 * h->kmax, ns), 256, h->bmax > 64 ? 0 : sfm::PSD_SMEM, st>>>(
                d_coef, h->d_coef_off + s0, h->d_b + s0, h->d_k + s0, d_nreg, pws, h->bmax);
        }
        BCK(h, cudaGetLastError());
        BCK(h, cudaMemcpyAsync(&nreg, d_nreg, sizeof(int), cudaMemcpyDeviceToHost, st));
        BCK(h, cudaStreamSynchronize(st));
        dfree(d_nreg);
    }
    rc = sfm::set_coeffs_device(h, d_coef);
    dfree(d_coef);
    if (rc) return rc;
    B->built = true;
    if (rep) {
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        rep->cg_iterations_max = cg_iters_max;
        rep->cg_residual_max = cg_res_max;
        rep->krylov_min_ratio = min_ratio;
        rep->nclasses = (int)B->classes.size();
        rep->nregularized = nreg;
    }
    return SFM_OK;
}

extern "C" int sfm_build_roms(sfm_handle* h, const int* m_sub, const int* k_sub, double sigma,
                              double cg_tol, sfm_build_report* rep) {
    return build_impl(h, m_sub, k_sub, sigma, cg_tol, rep, nullptr, nullptr);
}

extern "C" int sfm_build_roms_shifts(sfm_handle* h, const int* m_sub, const int* k_sub,
                                     const double* shifts, int nshifts, double cg_tol,
                                     sfm_build_report* rep) {
    if (!h) return SFM_ERR_ARG;
    BuildState* B = bstate(h);
    if (!B || !B->d_c) return bfail(h, SFM_ERR_STATE, "sfm_build_roms_shifts: no model");
    if (!m_sub || !k_sub || !shifts || nshifts < 0)
        return bfail(h, SFM_ERR_ARG, "sfm_build_roms_shifts: bad arguments");
    const int nsub = ((int)B->xc.size() - 1) * ((int)B->yc.size() - 1) * ((int)B->zc.size() - 1);
    int kmax = 1;
    for (int s = 0; s < nsub; ++s) kmax = std::max(kmax, k_sub[s]);
    if (nshifts < kmax - 1) return bfail(h, SFM_ERR_ARG, "sfm_build_roms_shifts: fewer shifts than kmax - 1");
    for (int i = 0; i < nshifts; ++i)
        if (!(shifts[i] > 0.0)) return bfail(h, SFM_ERR_ARG, "sfm_build_roms_shifts: shifts must be > 0");
    // the single-shift argument only has to be valid; every solve takes its
    // own shift
    return build_impl(h, m_sub, k_sub, nshifts > 0 ? shifts[0] : 1.0, cg_tol, rep, nullptr, nullptr,
                      shifts);
}

// Point weights of a set of points for every subdomain that holds one of
// their nodes: share M^a/M at shared nodes (Algorithm 1 step 1.4 reading).
// kind 0: Gaussian of the given width (cut at 3 widths, normalised);
// kind 1: trilinear interpolation.
static int project_points(sfm_handle* h, int npts, const double* xyz, int kind, double width,
                          std::vector<int>& pair_pt, std::vector<int>& pair_sub,
                          std::vector<double>& rows) {
    BuildState* B = bstate(h);
    const int ncx = (int)B->xc.size() - 1, ncy = (int)B->yc.size() - 1;
    const double hh = B->h;
    const int gx = B->gnx + 1, gy = B->gny + 1;
    // host node weights per point
    std::vector<std::vector<std::pair<long long, double>>> pw(npts);
    for (int p = 0; p < npts; ++p) {
        const double x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
        auto& w = pw[p];
        if (kind == 0) {
            const double rad = 3.0 * width;
            const int lo[3] = {std::max(0, (int)std::floor((x - rad) / hh)),
                               std::max(0, (int)std::floor((y - rad) / hh)),
                               std::max(0, (int)std::floor((z - rad) / hh))};
            const int hi[3] = {std::min(B->gnx, (int)std::ceil((x + rad) / hh)),
                               std::min(B->gny, (int)std::ceil((y + rad) / hh)),
                               std::min(B->gnz, (int)std::ceil((z + rad) / hh))};
            double tot = 0.0;
            for (int k = lo[2]; k <= hi[2]; ++k)
                for (int j = lo[1]; j <= hi[1]; ++j)
                    for (int i = lo[0]; i <= hi[0]; ++i) {
                        const double r2 = (i * hh - x) * (i * hh - x) + (j * hh - y) * (j * hh - y) +
                                          (k * hh - z) * (k * hh - z);
                        if (r2 > rad * rad + 1e-9 * hh * hh) continue;
                        const double v = std::exp(-r2 / (2.0 * width * width));
                        w.emplace_back(i + (long long)gx * (j + (long long)gy * k), v);
                        tot += v;
                    }
            for (auto& e : w) e.second /= tot;
        } else {
            const double f[3] = {x / hh, y / hh, z / hh};
            const int n[3] = {B->gnx, B->gny, B->gnz};
            int base[3];
            double fr[3];
            for (int a = 0; a < 3; ++a) {
                base[a] = std::max(0, std::min((int)std::floor(f[a] + 1e-12), n[a] - 1));
                fr[a] = std::min(1.0, std::max(0.0, f[a] - base[a]));
            }
            double tot = 0.0;
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const double v = (dx ? fr[0] : 1 - fr[0]) * (dy ? fr[1] : 1 - fr[1]) *
                                         (dz ? fr[2] : 1 - fr[2]);
                        if (v > 1e-14) {
                            w.emplace_back(base[0] + dx + (long long)gx * (base[1] + dy + (long long)gy * (base[2] + dz)), v);
                            tot += v;
                        }
                    }
            for (auto& e : w) e.second /= tot;
        }
    }
    // per class: pairs (point, subdomain in class) with node lists (local index, weight)
    cudaStream_t st = h->stream;
    const int nsub = (int)B->sub_class.size();
    std::vector<std::vector<std::tuple<int, int, std::vector<std::pair<int, double>>>>> per_class(B->classes.size());
    std::vector<std::pair<long long, int>> gidx;   // to fetch global masses
    for (int p = 0; p < npts; ++p) {
        std::map<int, std::vector<std::pair<int, double>>> by_sub;
        for (auto& e : pw[p]) {
            const long long g = e.first;
            const int i = (int)(g % gx), j = (int)((g / gx) % gy), k = (int)(g / ((long long)gx * gy));
            // subdomains whose closed box holds the node
            std::vector<int> sx, sy, sz;
            for (int a = 0; a < ncx; ++a) if (B->xc[a] <= i && i <= B->xc[a + 1]) sx.push_back(a);
            for (int a = 0; a < ncy; ++a) if (B->yc[a] <= j && j <= B->yc[a + 1]) sy.push_back(a);
            for (int a = 0; a < (int)B->zc.size() - 1; ++a) if (B->zc[a] <= k && k <= B->zc[a + 1]) sz.push_back(a);
            for (int a : sx) for (int bq : sy) for (int cq : sz) {
                const int s = a + ncx * (bq + ncy * cq);
                if (B->sub_class[s] < 0)
                    return bfail(h, SFM_ERR_STATE, "projection onto subdomain " + std::to_string(s) +
                                                       ", whose ROM came from the surrogate (no Krylov "
                                                       "basis): mark it exact");
                const BClass& c = B->classes[B->sub_class[s]];
                const int li = (i - B->xc[a]) + (c.nxl + 1) * ((j - B->yc[bq]) + (c.nyl + 1) * (k - B->zc[cq]));
                by_sub[s].emplace_back(li, e.second);
                (void)nsub;
            }
        }
        for (auto& kv : by_sub) {
            const int s = kv.first;
            per_class[B->sub_class[s]].emplace_back(p, s, kv.second);
        }
    }
    // global masses of the nodes involved: share = M^a / M
    std::vector<double> gm((size_t)gx * gy * (B->gnz + 1));
    BCK(h, cudaMemcpyAsync(gm.data(), B->d_gmass, gm.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    BCK(h, cudaStreamSynchronize(st));
    pair_pt.clear(); pair_sub.clear(); rows.clear();
    std::vector<std::tuple<int, int, std::vector<double>>> out;
    for (size_t ci = 0; ci < B->classes.size(); ++ci) {
        auto& pairs = per_class[ci];
        if (pairs.empty()) continue;
        const BClass& c = B->classes[ci];
        const int N = c.N, b = c.b, k = c.k, n = b * k, np = (int)pairs.size();
        // subdomain masses of this class (host copy, for the shares)
        std::vector<double> cm((size_t)c.subs.size() * N);
        BCK(h, cudaMemcpyAsync(cm.data(), c.mass, cm.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        BCK(h, cudaStreamSynchronize(st));
        std::vector<int> psub(np), nptr(np + 1, 0), nodes;
        std::vector<double> wts;
        for (int q = 0; q < np; ++q) {
            const int s = std::get<1>(pairs[q]);
            const int pos = B->sub_pos[s];
            psub[q] = pos;
            const int ix = s % ncx, iy = (s / ncx) % ncy, iz = s / (ncx * ncy);
            for (auto& e : std::get<2>(pairs[q])) {
                const int li = e.first;
                const int i = li % (c.nxl + 1), j = (li / (c.nxl + 1)) % (c.nyl + 1), kk = li / ((c.nxl + 1) * (c.nyl + 1));
                const long long g = (B->xc[ix] + i) + (long long)gx * ((B->yc[iy] + j) + (long long)gy * (B->zc[iz] + kk));
                nodes.push_back(li);
                wts.push_back(e.second * cm[(size_t)pos * N + li] / gm[g]);
            }
            nptr[q + 1] = (int)nodes.size();
        }
        int *d_psub = nullptr, *d_nptr = nullptr, *d_nodes = nullptr;
        double *d_w = nullptr, *Y = nullptr, *Z = nullptr, *R = nullptr;
        DevGuard guard_points(d_psub, d_nptr, d_nodes, d_w, Y, Z, R);
        BCK(h, dmalloc(d_psub, np));
        BCK(h, dmalloc(d_nptr, np + 1));
        BCK(h, dmalloc(d_nodes, nodes.size()));
        BCK(h, dmalloc(d_w, wts.size()));
        BCK(h, cudaMemcpyAsync(d_psub, psub.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
        BCK(h, cudaMemcpyAsync(d_nptr, nptr.data(), (np + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
        BCK(h, cudaMemcpyAsync(d_nodes, nodes.data(), nodes.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        BCK(h, cudaMemcpyAsync(d_w, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        BCK(h, dmalloc(Y, (size_t)np * n));
        BCK(h, dmalloc(Z, (size_t)np * n));
        BCK(h, dmalloc(R, (size_t)np * n));
        sfm::bld::gather_project_kernel<<<np, 256, 0, st>>>(c.V, c.mass, N, n, d_psub, d_nptr, d_nodes,
                                                            d_w, Y);
        BCK(h, cudaGetLastError());
        // Z = Qh^T Y per pair (one GEMV each; pairs are few)
        BuildState* BS = B;
        cublasSetStream(BS->blas, st);
        for (int q = 0; q < np; ++q) {
            const double one = 1.0, zero = 0.0;
            BLK(h, cublasDgemv(BS->blas, CUBLAS_OP_T, n, n, &one, c.Qh + (long long)psub[q] * n * n, n,
                               Y + (long long)q * n, 1, &zero, Z + (long long)q * n, 1));
        }
        sfm::bld::finish_project_kernel<<<np, 256, 0, st>>>(Z, c.Ginv, b, k, d_psub, R);
        BCK(h, cudaGetLastError());
        std::vector<double> hr((size_t)np * n);
        BCK(h, cudaMemcpyAsync(hr.data(), R, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        BCK(h, cudaStreamSynchronize(st));
        for (int q = 0; q < np; ++q)
            out.emplace_back(std::get<0>(pairs[q]), std::get<1>(pairs[q]),
                             std::vector<double>(hr.begin() + (size_t)q * n, hr.begin() + (size_t)(q + 1) * n));
        for (int** p : {&d_psub, &d_nptr, &d_nodes}) dfree(*p);
        for (double** p : {&d_w, &Y, &Z, &R}) dfree(*p);
    }
    std::sort(out.begin(), out.end(), [](const auto& a, const auto& b) {
        return std::make_pair(std::get<0>(a), std::get<1>(a)) < std::make_pair(std::get<0>(b), std::get<1>(b));
    });
    for (auto& e : out) {
        pair_pt.push_back(std::get<0>(e));
        pair_sub.push_back(std::get<1>(e));
        rows.insert(rows.end(), std::get<2>(e).begin(), std::get<2>(e).end());
    }
    return SFM_OK;
}

extern "C" int sfm_free_build(sfm_handle* h) {
    if (!h) return SFM_ERR_ARG;
    BuildState* B = bstate(h);
    if (B) {
        cudaSetDevice(h->device);
        cudaStreamSynchronize(h->stream);
        free_classes(B);
    }
    return SFM_OK;
}

extern "C" int sfm_project_sources(sfm_handle* h, int nshots, const double* xyz, double width) {
    if (!h) return SFM_ERR_ARG;
    BuildState* B = bstate(h);
    if (!B || !B->built) return bfail(h, SFM_ERR_STATE, "sfm_project_sources: no ROMs built");
    if (nshots < 1 || !xyz || !(width > 0.0)) return bfail(h, SFM_ERR_ARG, "sfm_project_sources: bad arguments");
    BCK(h, cudaSetDevice(h->device));
    std::vector<int> pp, ps;
    std::vector<double> rows;
    int rc = project_points(h, nshots, xyz, 0, width, pp, ps, rows);
    if (rc) return rc;
    return sfm_set_sources(h, nshots, (int)pp.size(), pp.data(), ps.data(), rows.data());
}

extern "C" int sfm_project_receivers(sfm_handle* h, int nrec, const double* xyz) {
    if (!h) return SFM_ERR_ARG;
    BuildState* B = bstate(h);
    if (!B || !B->built) return bfail(h, SFM_ERR_STATE, "sfm_project_receivers: no ROMs built");
    if (nrec < 1 || !xyz) return bfail(h, SFM_ERR_ARG, "sfm_project_receivers: bad arguments");
    BCK(h, cudaSetDevice(h->device));
    std::vector<int> pp, ps;
    std::vector<double> rows;
    int rc = project_points(h, nrec, xyz, 1, 0.0, pp, ps, rows);
    if (rc) return rc;
    return sfm_set_receivers(h, nrec, (int)pp.size(), pp.data(), ps.data(), rows.data());
}

// ---------------------------------------------------------------------------
// Surrogate mode of the offline stage
// ---------------------------------------------------------------------------
namespace {

// velocity blocks of S subdomains of n^3 cells (origins in cells) as FP32
__global__ void gather_blocks_kernel(const double* c, int gnx, int gny, const int3* origin, int S, int n,
                                     float* out) {
    const long long n3 = (long long)n * n * n, total = (long long)S * n3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / n3);
        const long long e = t - s * n3;
        const int x = (int)(e % n), y = (int)((e / n) % n), z = (int)(e / ((long long)n * n));
        const int3 o = origin[s];
        out[t] = (float)c[((long long)(o.z + z) * gny + (o.y + y)) * gnx + (o.x + x)];
    }
}

// Gamma_1 into level 0 (symmetrised) and Gammahat_1 into level k of each set
__global__ void put_level1_kernel(const double* G1, const double* Gh1, int S, int b, int k, double* sets) {
    const long long bb = (long long)b * b, total = (long long)S * bb;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / bb);
        const int e = (int)(t - s * bb), r = e / b, c = e % b;
        double* set = sets + (long long)s * 2 * k * bb;
        set[e] = 0.5 * (G1[s * bb + r * b + c] + G1[s * bb + c * b + r]);
        set[k * bb + e] = 0.5 * (Gh1[s * bb + r * b + c] + Gh1[s * bb + c * b + r]);
    }
}

}  // namespace

extern "C" int sfm_build_roms_surrogate(sfm_handle* h, sfm_net* net, const int* m_sub, const int* k_sub,
                                        double sigma, double cg_tol, double nt_tol, const int* exact,
                                        sfm_surrogate_report* srep, sfm_build_report* rep) {
    if (!h) return SFM_ERR_ARG;
    BuildState* B = bstate(h);
    if (!B || !B->d_c) return bfail(h, SFM_ERR_STATE, "sfm_build_roms_surrogate: no model");
    if (!net || !m_sub || !k_sub || !(sigma > 0.0) || !(nt_tol >= 0.0))
        return bfail(h, SFM_ERR_ARG, "sfm_build_roms_surrogate: bad arguments");
    int nn = 0, nb = 0, nk = 0;
    if (sfm::net_shape(net, &nn, &nb, &nk) != SFM_OK)
        return bfail(h, SFM_ERR_STATE, "sfm_build_roms_surrogate: the network has no decoder");
    if (!(cg_tol > 0.0)) cg_tol = 1e-14;
    BCK(h, cudaSetDevice(h->device));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = h->stream;
    cublasSetStream(B->blas, st);
    cublasSetPointerMode(B->blas, CUBLAS_POINTER_MODE_HOST);
    const Gemm gemm{B->blas};
    const int ncx = (int)B->xc.size() - 1, ncy = (int)B->yc.size() - 1, ncz = (int)B->zc.size() - 1;
    const int nsub = ncx * ncy * ncz;
    // topology as the exact build forms it (coefficient layout for the presets)
    std::vector<int> nbr(6 * nsub, -1), mface(6 * nsub, 0);
    for (int s = 0; s < nsub; ++s) {
        if (k_sub[s] < 1 || m_sub[s] < 1) return bfail(h, SFM_ERR_ARG, "sfm_build_roms_surrogate: m, k >= 1");
        const int pos[3] = {s % ncx, (s / ncx) % ncy, s / (ncx * ncy)};
        const int lim[3] = {ncx, ncy, ncz};
        for (int f = 0; f < 6; ++f) {
            int q[3] = {pos[0], pos[1], pos[2]};
            q[f / 2] += (f & 1) ? 1 : -1;
            if (q[f / 2] >= 0 && q[f / 2] < lim[f / 2]) nbr[s * 6 + f] = q[0] + ncx * (q[1] + ncy * q[2]);
        }
    }
    for (int s = 0; s < nsub; ++s)
        for (int f = 0; f < 6; ++f) {
            const int t = nbr[s * 6 + f];
            mface[s * 6 + f] = (t < 0) ? m_sub[s] : std::min(m_sub[s], m_sub[t]);
        }
    int rc = sfm::set_topology_internal(h, nsub, k_sub, mface.data(), nbr.data());
    if (rc != SFM_OK) return rc;
    // subdomains the network can serve: n^3 cells, k levels, the decoder's b
    // with the same m on all six faces, and not marked exact by the caller
    std::vector<int> elig;
    std::vector<int3> org;
    const int m = nb / 6;
    for (int s = 0; s < nsub; ++s) {
        const int ix = s % ncx, iy = (s / ncx) % ncy, iz = s / (ncx * ncy);
        bool ok = (!exact || !exact[s]) && k_sub[s] == nk && nb % 6 == 0 &&
                  B->xc[ix + 1] - B->xc[ix] == nn && B->yc[iy + 1] - B->yc[iy] == nn &&
                  B->zc[iz + 1] - B->zc[iz] == nn;
        for (int f = 0; f < 6 && ok; ++f) ok = mface[s * 6 + f] == m;
        if (ok) {
            elig.push_back(s);
            org.push_back(make_int3(B->xc[ix], B->yc[iy], B->zc[iz]));
        }
    }
    const int S = (int)elig.size();
    std::vector<char> only(nsub, 1);
    std::vector<double> herr(S, 0.0);
    double* d_preset = nullptr;
    DevGuard guard_preset(d_preset);
    BCK(h, dmalloc(d_preset, (size_t)h->ncoef));
    BCK(h, cudaMemsetAsync(d_preset, 0, (size_t)h->ncoef * sizeof(double), st));
    int naccept = 0;
    if (S > 0) {
        const int b = nb, k = nk, N = (nn + 1) * (nn + 1) * (nn + 1);
        const long long bb = (long long)b * b, sF = (long long)N * b;
        int3* d_org = nullptr;
        double *mass = nullptr, *Bm = nullptr, *F = nullptr, *LF = nullptr, *Gh1 = nullptr, *R0 = nullptr,
               *R0i = nullptr, *Gi = nullptr, *A1 = nullptr, *T1 = nullptr, *G1 = nullptr, *Ss = nullptr,
               *sets = nullptr, *d_err2 = nullptr, *serr = nullptr;
        float *blocks = nullptr, *codes = nullptr;
        ColSpec* d_cs = nullptr;
        int* d_e = nullptr;
        DevGuard g1(d_org);
        DevGuard g2(mass, Bm, F, LF, Gh1, R0, R0i, Gi, A1, T1, G1, Ss, sets, d_err2, serr);
        DevGuard g3(blocks, codes);
        DevGuard g4(d_cs);
        DevGuard g5(d_e);
        BCK(h, dmalloc(d_org, S));
        BCK(h, cudaMemcpyAsync(d_org, org.data(), S * sizeof(int3), cudaMemcpyHostToDevice, st));
        BCK(h, dmalloc(mass, (size_t)S * N));
        sfm::bld::mass_kernel<<<grid_for((long long)S * N), 256, 0, st>>>(B->d_c, B->gnx, B->gny, d_org, S,
                                                                            nn, nn, nn, B->h, mass);
        std::vector<ColSpec> cs;
        for (int f = 0; f < 6; ++f)
            for (auto pq : face_modes(nn - 1, nn - 1, m)) cs.push_back({f, pq.first, pq.second, 0});
        BCK(h, dmalloc(d_cs, cs.size()));
        BCK(h, cudaMemcpyAsync(d_cs, cs.data(), cs.size() * sizeof(ColSpec), cudaMemcpyHostToDevice, st));
        BCK(h, dmalloc(Bm, (size_t)N * b));
        sfm::bld::basis_kernel<<<grid_for((long long)N * b), 256, 0, st>>>(d_cs, b, nn, nn, nn, B->h, Bm);
        // F = M^{-1/2} B
        BCK(h, dmalloc(F, (size_t)S * sF));
        sfm::bld::scale_kernel<<<grid_for((long long)S * sF), 256, 0, st>>>(Bm, 0, mass, F, sF, N, b, S, 1);
        BCK(h, cudaGetLastError());
        // level 1 closed forms: Gammahat_1 = F^T F, Gamma_1 = G^{-1} F^T L F G^{-1}
        for (double** p : {&Gh1, &R0, &R0i, &Gi, &A1, &T1, &G1, &Ss}) BCK(h, dmalloc(*p, (size_t)S * bb));
        BLK(h, gemm(true, false, b, b, N, 1.0, F, N, sF, F, N, sF, 0.0, Gh1, b, bb, S));
        BCK(h, dmalloc(d_e, 1));
        BCK(h, cudaMemsetAsync(d_e, 0, sizeof(int), st));
        BCK(h, dmalloc(d_err2, (size_t)S));
        const size_t csm = 2 * bb * sizeof(double);
        BCK(h, cudaFuncSetAttribute(sfm::bld::chol_rinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)csm));
        sfm::bld::chol_rinv_kernel<<<S, 128, csm, st>>>(Gh1, R0, R0i, b, d_e, d_err2, nullptr);
        BCK(h, cudaGetLastError());
        BLK(h, gemm(false, true, b, b, b, 1.0, R0i, b, bb, R0i, b, bb, 0.0, Gi, b, bb, S));   // (F^T F)^{-1}
        BCK(h, dmalloc(LF, (size_t)S * sF));
        sfm::bld::op_kernel<<<S * b, 256, 0, st>>>(F, LF, mass, nn, nn, nn, B->h, 0.0, b, 1, nullptr);
        BCK(h, cudaGetLastError());
        BLK(h, gemm(true, false, b, b, N, 1.0, F, N, sF, LF, N, sF, 0.0, A1, b, bb, S));      // F^T L F
        BLK(h, gemm(false, false, b, b, b, 1.0, Gi, b, bb, A1, b, bb, 0.0, T1, b, bb, S));
        BLK(h, gemm(false, false, b, b, b, 1.0, T1, b, bb, Gi, b, bb, 0.0, G1, b, bb, S));
        // one block solve: S(sigma) = F^T (L + sigma)^{-1} F, CG on (K + sigma M)
        {
            const size_t ncolv = (size_t)S * b;
            double *Xc = nullptr, *Rc = nullptr, *Zc = nullptr, *Pc = nullptr, *Qc = nullptr, *rhs = nullptr,
                   *rz = nullptr, *rz2 = nullptr, *pq = nullptr, *rr = nullptr, *rr0 = nullptr;
            DevGuard guard_cg(Xc, Rc, Zc, Pc, Qc, rhs, rz, rz2, pq, rr, rr0);
            for (double** p : {&Xc, &Rc, &Zc, &Pc, &Qc, &rhs}) BCK(h, dmalloc(*p, ncolv * N));
            for (double** p : {&rz, &rz2, &pq, &rr, &rr0}) BCK(h, dmalloc(*p, ncolv));
            sfm::bld::scale_kernel<<<grid_for((long long)ncolv * N), 256, 0, st>>>(F, sF, mass, rhs, sF, N, b, S, 0);
            sfm::bld::cg_init_kernel<<<(int)ncolv, 256, 0, st>>>(rhs, Xc, Rc, Zc, Pc, mass, nn, nn, nn, B->h,
                                                                 sigma, b, rz, rr0);
            BCK(h, cudaGetLastError());
            std::vector<double> h_rr(ncolv), h_rr0(ncolv);
            BCK(h, cudaMemcpyAsync(h_rr0.data(), rr0, ncolv * sizeof(double), cudaMemcpyDeviceToHost, st));
            int it = 0;
            for (it = 1; it <= 20000; ++it) {
                sfm::bld::op_kernel<<<(int)ncolv, 256, 0, st>>>(Pc, Qc, mass, nn, nn, nn, B->h, sigma, b, 0, pq);
                sfm::bld::cg_update_kernel<<<(int)ncolv, 256, 0, st>>>(Xc, Rc, Zc, Pc, Qc, mass, nn, nn, nn, B->h,
                                                                       sigma, b, rz, pq, rz2, rr);
                sfm::bld::cg_dir_kernel<<<(int)ncolv, 256, 0, st>>>(Pc, Zc, N, rz, rz2);
                if (it % 8 == 0) {
                    BCK(h, cudaGetLastError());
                    BCK(h, cudaMemcpyAsync(h_rr.data(), rr, ncolv * sizeof(double), cudaMemcpyDeviceToHost, st));
                    BCK(h, cudaStreamSynchronize(st));
                    double worst = 0.0;
                    for (size_t i = 0; i < ncolv; ++i)
                        if (h_rr0[i] > 0) worst = std::max(worst, std::sqrt(h_rr[i] / h_rr0[i]));
                    if (worst < cg_tol) break;
                }
            }
            if (it > 20000) return bfail(h, SFM_ERR_BREAKDOWN, "sfm_build_roms_surrogate: CG did not converge");
            // W = M^{1/2} Y into LF, S(sigma) = F^T W
            sfm::bld::scale_kernel<<<grid_for((long long)ncolv * N), 256, 0, st>>>(Xc, sF, mass, LF, sF, N, b, S, 0);
            BCK(h, cudaGetLastError());
            BLK(h, gemm(true, false, b, b, N, 1.0, F, N, sF, LF, N, sF, 0.0, Ss, b, bb, S));
            // S'(sigma) = -F^T (L + sigma)^{-2} F = -W^T W from the same solve
            BLK(h, gemm(true, false, b, b, N, -1.0, LF, N, sF, LF, N, sF, 0.0, A1, b, bb, S));
        }
        // the network's coefficient sets: levels 2..k decoded, level 1 exact
        BCK(h, dmalloc(blocks, (size_t)S * nn * nn * nn));
        gather_blocks_kernel<<<grid_for((long long)S * nn * nn * nn), 256, 0, st>>>(B->d_c, B->gnx, B->gny, d_org,
                                                                                    S, nn, blocks);
        BCK(h, cudaGetLastError());
        BCK(h, cudaStreamSynchronize(st));
        BCK(h, dmalloc(sets, (size_t)S * 2 * k * bb));
        BCK(h, cudaMemsetAsync(sets, 0, (size_t)S * 2 * k * bb * sizeof(double), st));
        BCK(h, cudaStreamSynchronize(st));
        const int ncode = sfm::net_code_dim(net);
        BCK(h, dmalloc(codes, (size_t)S * ncode));
        rc = sfm_net_forward(net, blocks, S, codes, 1);
        if (rc != SFM_OK) return bfail(h, rc, std::string("sfm_build_roms_surrogate: network: ") + sfm_net_last_error(net));
        rc = sfm_net_decode(net, codes, S, sets);
        if (rc != SFM_OK) return bfail(h, rc, std::string("sfm_build_roms_surrogate: decoder: ") + sfm_net_last_error(net));
        put_level1_kernel<<<grid_for((long long)S * bb), 256, 0, st>>>(G1, Gh1, S, b, k, sets);
        BCK(h, cudaGetLastError());
        // fallback test at sigma
        BCK(h, dmalloc(serr, (size_t)S));
        BCK(h, sfm::sigma_check(sets, S, b, k, sigma, Ss, A1, serr, st));
        BCK(h, cudaMemcpy(herr.data(), serr, S * sizeof(double), cudaMemcpyDeviceToHost));
        for (int i = 0; i < S; ++i) {
            const int s = elig[i];
            if (herr[i] <= nt_tol) {
                only[s] = 0;
                ++naccept;
                BCK(h, cudaMemcpyAsync(d_preset + h->coef_off[s], sets + (long long)i * 2 * k * bb,
                                       2 * k * bb * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
        }
        BCK(h, cudaStreamSynchronize(st));
    }
    const double t_sur = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const auto t1 = std::chrono::steady_clock::now();
    rc = build_impl(h, m_sub, k_sub, sigma, cg_tol, rep, naccept > 0 ? &only : nullptr, d_preset);
    if (rc != SFM_OK) return rc;
    if (srep) {
        srep->eligible = S;
        srep->accepted = naccept;
        srep->fallback = S - naccept;
        std::vector<double> acc;
        for (int i = 0; i < S; ++i)
            if (herr[i] <= nt_tol) acc.push_back(herr[i]);
        std::sort(herr.begin(), herr.end());
        srep->sigma_err_median = S ? herr[S / 2] : 0.0;
        srep->sigma_err_max_accepted = acc.empty() ? 0.0 : *std::max_element(acc.begin(), acc.end());
        srep->seconds_surrogate = t_sur;
        srep->seconds_exact = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
    }
    return SFM_OK;
}
