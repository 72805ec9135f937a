// Usable depth of every subdomain's S-fraction, and the cut to it.
//
// An extension of the offline stage (the paper's own ROMs are three levels
// deep).  The deep levels of an accurate ROM at a small shift run past
// FP64's dynamic range: the smallest eigenvalues of their Gamma_j and
// Gammahat_j (Eq. 13) sit at the rounding level, some rounded below zero,
// and the coupled stability limit of the fraction falls far below the
// Galerkin ROM's.  A fraction cut after level d and terminated with
// U_{d+1} = 0, like the full one (Eq. 12), is a positive definite
// S-fraction of order d; its source, receiver and initial rows are the
// first d levels of the full ones.
#include "sfm_internal.h"

#include <algorithm>
#include <vector>

namespace {

constexpr int RLD = 65;      // leading dimension of the shared block (bank spread)

// Extreme eigenvalues of every block (Gamma_1..k, then Gammahat_1..k) of
// every subdomain: cyclic Jacobi rotations on the symmetrised block in
// shared memory, one block of threads per matrix, at most 30 sweeps (each a
// fixed number of rotations), stopped once the off-diagonal mass is below
// 1e-30 of the diagonal's (squared sums).  range[(s*2*kmax + blk)*2 + 0/1]
// = (lambda_min, lambda_max); blocks beyond 2 k_s are left untouched.
__global__ void __launch_bounds__(256) block_range_kernel(const double* coef,
                                                          const long long* coef_off,
                                                          const int* sub_b, const int* sub_k,
                                                          int kmax, double* range) {
    __shared__ double A[64 * RLD];
    __shared__ double s_cs[2];
    __shared__ int s_done;
    const int s = blockIdx.y, blk = blockIdx.x;
    const int b = sub_b[s], k = sub_k[s];
    if (blk >= 2 * k) return;
    const double* m = coef + coef_off[s] + (long long)blk * b * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        A[i * RLD + j] = 0.5 * (m[i * b + j] + m[j * b + i]);
    }
    __syncthreads();
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (threadIdx.x == 0) {
            double off = 0.0, dia = 0.0;
            for (int i = 0; i < b; ++i)
                for (int j = 0; j < b; ++j)
                    (i == j ? dia : off) += A[i * RLD + j] * A[i * RLD + j];
            s_done = (off <= 1e-30 * dia) ? 1 : 0;
        }
        __syncthreads();
        if (s_done) break;
        for (int pp = 0; pp < b - 1; ++pp) {
            for (int qq = pp + 1; qq < b; ++qq) {
                if (threadIdx.x == 0) {
                    // rotation that zeroes A[pp][qq]: t = tan of its angle,
                    // the root of t^2 + 2 theta t - 1 = 0 of smaller modulus
                    const double apq = A[pp * RLD + qq];
                    double c = 1.0, sn = 0.0;
                    if (apq != 0.0) {
                        const double theta = (A[qq * RLD + qq] - A[pp * RLD + pp]) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) /
                                         (fabs(theta) + sqrt(1.0 + theta * theta));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                    }
                    s_cs[0] = c;
                    s_cs[1] = sn;
                }
                __syncthreads();
                const double c = s_cs[0], sn = s_cs[1];
                if (sn != 0.0) {
                    for (int i = threadIdx.x; i < b; i += blockDim.x) {
                        const double aip = A[i * RLD + pp], aiq = A[i * RLD + qq];
                        A[i * RLD + pp] = c * aip - sn * aiq;
                        A[i * RLD + qq] = sn * aip + c * aiq;
                    }
                    __syncthreads();
                    for (int j = threadIdx.x; j < b; j += blockDim.x) {
                        const double apj = A[pp * RLD + j], aqj = A[qq * RLD + j];
                        A[pp * RLD + j] = c * apj - sn * aqj;
                        A[qq * RLD + j] = sn * apj + c * aqj;
                    }
                }
                __syncthreads();
            }
        }
    }
    if (threadIdx.x == 0) {
        double lo = A[0], hi = A[0];
        for (int t = 1; t < b; ++t) {
            lo = fmin(lo, A[t * RLD + t]);
            hi = fmax(hi, A[t * RLD + t]);
        }
        double* out = range + ((long long)s * 2 * kmax + blk) * 2;
        out[0] = lo;
        out[1] = hi;
    }
}

}  // namespace

extern "C" {

int sfm_usable_depths(int nsub, const int* k_sub, int kmax, const double* range, double tau,
                      int* depth) {
    if (nsub < 1 || !k_sub || kmax < 1 || !range || !depth || !(tau >= 0.0 && tau < 1.0)) {
        sfm::set_global_error("sfm_usable_depths: bad arguments");
        return SFM_ERR_ARG;
    }
    for (int s = 0; s < nsub; ++s) {
        const int k = k_sub[s];
        if (k < 1 || k > kmax) {
            sfm::set_global_error("sfm_usable_depths: k out of range");
            return SFM_ERR_ARG;
        }
        const double* r = range + (size_t)s * 2 * kmax * 2;
        int d = k;
        for (int j = 0; j < k; ++j) {
            const double* gh = r + (size_t)(k + j) * 2;      // Gammahat_{j+1}
            bool ok = gh[0] > tau * gh[1];
            if (j < k - 1) {                                 // Gamma_k is semidefinite
                const double* g = r + (size_t)j * 2;
                ok = ok && g[0] > tau * g[1];
            }
            if (!ok) {
                d = std::max(j, 1);
                break;
            }
        }
        depth[s] = d;
    }
    return SFM_OK;
}

int sfm_cut_depth(sfm_handle* h, double tau, int* depth_out, int depth_cap, int* nlevels_cut) {
    if (!h) {
        sfm::set_global_error("NULL handle");
        return SFM_ERR_ARG;
    }
    if (!(tau >= 0.0 && tau < 1.0)) {
        h->err = "sfm_cut_depth: tau must be in [0, 1)";
        return SFM_ERR_ARG;
    }
    if (h->nsub == 0 || !h->have_coef) {
        h->err = "sfm_cut_depth: no coefficients";
        return SFM_ERR_STATE;
    }
    if (h->bmax > sfm::BMAX_NARROW) {
        h->err = "sfm_cut_depth: blocks wider than 64 (its eigenvalue ranges work in 64-wide shared memory)";
        return SFM_ERR_ARG;
    }
    if (depth_out && depth_cap < h->nsub) {
        h->err = "sfm_cut_depth: depth_out holds fewer than nsub entries";
        return SFM_ERR_ARG;
    }
    const int nsub = h->nsub, kmax = h->kmax;
    cudaStream_t st = h->stream;
    auto cuda_err = [&](cudaError_t e, const char* what) {
        h->err = std::string("sfm_cut_depth: ") + what + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SFM_ERR_NOMEM : SFM_ERR_CUDA;
    };
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_err(e, "cudaSetDevice");

    // extreme eigenvalues of every block, on the device
    std::vector<double> range((size_t)nsub * 2 * kmax * 2, 0.0);
    {
        double* d_range = nullptr;
        e = cudaMalloc((void**)&d_range, range.size() * sizeof(double));
        if (e != cudaSuccess) return cuda_err(e, "cudaMalloc");
        for (int s0 = 0; s0 < nsub && e == cudaSuccess; s0 += 65535) {
            const int ns = std::min(65535, nsub - s0);
            block_range_kernel<<<dim3(2 * kmax, ns), 256, 0, st>>>(
                h->d_coef64, h->d_coef_off + s0, h->d_b + s0, h->d_k + s0, kmax,
                d_range + (size_t)s0 * 2 * kmax * 2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(range.data(), d_range, range.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(d_range);
        if (e != cudaSuccess) return cuda_err(e, "block eigenvalue ranges");
    }
    std::vector<int> depth(nsub);
    int rc = sfm_usable_depths(nsub, h->k.data(), kmax, range.data(), tau, depth.data());
    if (rc != SFM_OK) {
        h->err = "sfm_cut_depth: depth decision failed";
        return rc;
    }
    int ncut = 0;
    for (int s = 0; s < nsub; ++s) ncut += h->k[s] - depth[s];
    if (depth_out) std::copy(depth.begin(), depth.end(), depth_out);
    if (nlevels_cut) *nlevels_cut = ncut;
    if (ncut == 0) return SFM_OK;

    // host copies of everything laid out by level, then the cut layout set
    // through the ordinary entry points
    const std::vector<int> k_old = h->k, b = h->b, mface = h->mface, nbr = h->nbr;
    const std::vector<long long> coef_off = h->coef_off, state_off = h->state_off;
    auto d2h = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
    };
    std::vector<double> coef((size_t)h->ncoef);
    e = d2h(coef.data(), h->d_coef64, coef.size() * sizeof(double));
    const bool had_src = h->have_src, had_rec = h->have_rec, had_init = h->have_init;
    std::vector<double> src, rrows, U0, V0;
    if (e == cudaSuccess && had_src) {
        src.resize((size_t)h->nsrc);
        e = d2h(src.data(), h->d_src64, src.size() * sizeof(double));
    }
    if (e == cudaSuccess && had_rec) {
        rrows.resize((size_t)h->nrrow);
        e = d2h(rrows.data(), h->d_rrows64, rrows.size() * sizeof(double));
    }
    const bool had_v0 = had_init && h->d_init_V64 != nullptr;
    const bool had_delta = had_init && h->init_delta;    // a state from sfm_restore
    if (e == cudaSuccess && had_init) {
        U0.resize((size_t)h->init_nshots * h->nstate);
        e = d2h(U0.data(), h->d_init_U64, U0.size() * sizeof(double));
        if (e == cudaSuccess && had_v0) {
            V0.resize(U0.size());
            e = d2h(V0.data(), h->d_init_V64, V0.size() * sizeof(double));
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "copy to the host");

    // coefficients: Gamma_1..d then Gammahat_1..d of every subdomain
    std::vector<double> coef_new;
    for (int s = 0; s < nsub; ++s) {
        const size_t bb = (size_t)b[s] * b[s];
        const double* base = coef.data() + coef_off[s];
        coef_new.insert(coef_new.end(), base, base + depth[s] * bb);
        coef_new.insert(coef_new.end(), base + k_old[s] * bb, base + (k_old[s] + depth[s]) * bb);
    }
    // per (shot, subdomain) source pairs in their stored order
    const int nshots = h->nshots;
    std::vector<int> src_shot, src_sub;
    std::vector<double> src_new;
    if (had_src) {
        std::vector<std::pair<long long, int>> order;
        for (size_t i = 0; i < h->src_off.size(); ++i)
            if (h->src_off[i] >= 0) order.push_back({h->src_off[i], (int)i});
        std::sort(order.begin(), order.end());
        for (auto& o : order) {
            const int q = o.second / nsub, s = o.second % nsub;
            src_shot.push_back(q);
            src_sub.push_back(s);
            const double* row = src.data() + o.first;
            src_new.insert(src_new.end(), row, row + (size_t)depth[s] * b[s]);
        }
    }
    const int nrec = h->nrec;
    std::vector<int> rec_id, rec_sub;
    std::vector<double> rec_new;
    if (had_rec) {
        for (int i = 0; i < h->nrpairs; ++i) {
            const int s = h->rp_sub[i];
            rec_id.push_back(h->rp_rec[i]);
            rec_sub.push_back(s);
            const double* row = rrows.data() + h->rp_off[i];
            rec_new.insert(rec_new.end(), row, row + (size_t)depth[s] * b[s]);
        }
    }
    const int init_nshots = h->init_nshots;
    std::vector<int> ini_shot, ini_sub;
    std::vector<double> U0_new, V0_new;
    if (had_init) {
        const size_t nstate = (size_t)h->nstate;
        for (int q = 0; q < init_nshots; ++q)
            for (int s = 0; s < nsub; ++s) {
                ini_shot.push_back(q);
                ini_sub.push_back(s);
                const size_t at = q * nstate + state_off[s];
                U0_new.insert(U0_new.end(), U0.begin() + at, U0.begin() + at + (size_t)depth[s] * b[s]);
                if (had_v0)
                    V0_new.insert(V0_new.end(), V0.begin() + at,
                                  V0.begin() + at + (size_t)depth[s] * b[s]);
            }
    }

    // the offline bases describe the uncut fraction: projecting with them
    // after the cut would give rows of the wrong depth, so they are released
    // (the velocity model stays for a new sfm_build_roms)
    if ((rc = sfm_free_build(h)) != SFM_OK) return rc;
    if ((rc = sfm_set_topology(h, nsub, depth.data(), mface.data(), nbr.data())) != SFM_OK) return rc;
    if ((rc = sfm_set_coeffs(h, coef_new.data(), coef_new.size())) != SFM_OK) return rc;
    if (had_src && (rc = sfm_set_sources(h, nshots, (int)src_sub.size(), src_shot.data(),
                                         src_sub.data(), src_new.data())) != SFM_OK)
        return rc;
    if (had_rec && (rc = sfm_set_receivers(h, nrec, (int)rec_sub.size(), rec_id.data(),
                                           rec_sub.data(), rec_new.data())) != SFM_OK)
        return rc;
    if (had_init && (rc = sfm_set_initial(h, init_nshots, (int)ini_sub.size(), ini_shot.data(),
                                          ini_sub.data(), U0_new.data(),
                                          had_v0 ? V0_new.data() : nullptr)) != SFM_OK)
        return rc;
    h->init_delta = had_delta;      // a restored increment stays an increment
    return SFM_OK;
}

}  // extern "C"
