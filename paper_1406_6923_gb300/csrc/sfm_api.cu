// Host side of the libsfm C ABI: handle, topology, coefficient/source/
// receiver upload, precision caches and the stepping driver.
#include "sfm_internal.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <new>

namespace {

thread_local std::string g_err;

int fail(sfm_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg; else g_err = msg;
    return code;
}

int cuda_fail(sfm_handle* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, SFM_ERR_NOMEM, m);
    return fail(h, SFM_ERR_CUDA, m);
}

#define CK(h, call)                                              \
    do {                                                         \
        cudaError_t e__ = (call);                                \
        if (e__ != cudaSuccess) return cuda_fail((h), e__, #call); \
    } while (0)

template <typename P>
void dfree(P*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

template <typename P>
cudaError_t dalloc(P*& p, size_t count) {
    dfree(p);
    if (count == 0) count = 1;
    return cudaMalloc((void**)&p, count * sizeof(P));
}

template <typename P>
cudaError_t upload(P*& d, const P* host, size_t count, cudaStream_t st) {
    cudaError_t e = dalloc(d, count);
    if (e != cudaSuccess) return e;
    if (count) e = cudaMemcpyAsync(d, host, count * sizeof(P), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

// Converted copies of the FP64 master data in one compute precision.
template <typename T>
struct Cache {
    T *coef = nullptr, *H = nullptr, *src = nullptr, *rrows = nullptr;
    float* fcoef = nullptr;            // factored policies: FP32 factor tiles (coef unused)
    bool valid = false;
    void release() {
        dfree(coef); dfree(fcoef); dfree(H); dfree(src); dfree(rrows);
        valid = false;
    }
};

// Run buffers in one precision, grown on demand.
template <typename T>
struct RunBufs {
    T *U[4] = {nullptr, nullptr, nullptr, nullptr}, *dU = nullptr, *mail[2] = {nullptr, nullptr};
    T *wavelet = nullptr, *partial = nullptr;
    unsigned* rctr = nullptr;
    size_t n_state = 0, n_mail = 0, n_wav = 0, n_part = 0, n_ctr = 0;
    void release() {
        for (auto& u : U) dfree(u);
        dfree(dU); dfree(mail[0]); dfree(mail[1]); dfree(wavelet); dfree(partial); dfree(rctr);
        n_state = n_mail = n_wav = n_part = n_ctr = 0;
    }
};

}  // namespace

namespace sfm {
void set_global_error(const std::string& msg) { g_err = msg; }
}  // namespace sfm

// Data of the multi-shot panel modes (panel.cu), all FP32: padded factor
// tiles, face blocks, source panels per (group, subdomain) unit, receiver
// rows, and the per-subdomain receiver pair lists.
struct PanelCache {
    float *coef = nullptr, *H = nullptr, *src = nullptr, *rrows = nullptr;
    long long *d_coef_off = nullptr, *d_src_off = nullptr;
    // two-float mode: padded two-float tiles of the symmetric blocks, their
    // per-subdomain offsets (floats) and H_f as (hi, lo) pairs, built on
    // first use
    float *coef2 = nullptr, *H2 = nullptr, *rrows2 = nullptr;
    long long* d_coef2_off = nullptr;
    int *d_sub_rp_ptr = nullptr, *d_sub_rp = nullptr;
    int ngroups = 0, rpmax = 0;
    bool valid = false;
    void release() {
        dfree(coef); dfree(H); dfree(src); dfree(rrows);
        dfree(d_coef_off); dfree(d_src_off); dfree(d_sub_rp_ptr); dfree(d_sub_rp);
        dfree(coef2); dfree(H2); dfree(rrows2); dfree(d_coef2_off);
        ngroups = rpmax = 0;
        valid = false;
    }
};

struct PanelBufs {
    float *U = nullptr, *dU = nullptr, *mail[2] = {nullptr, nullptr}, *wav = nullptr,
          *partial = nullptr;
    size_t n_state = 0, n_mail = 0, n_wav = 0, n_part = 0;
    void release() {
        dfree(U); dfree(dU); dfree(mail[0]); dfree(mail[1]); dfree(wav); dfree(partial);
        n_state = n_mail = n_wav = n_part = 0;
    }
};

struct sfm_ext {
    // report of the last sfm_run (sfm_run_report)
    sfm_run_info info{-1, 0, 0, 0, 0.0, 0.0, 0, -1, 0};
    std::vector<double> energy;        // E^{-1/2} then E^{N-1/2}, per shot
    int* d_ustep = nullptr;            // instability sentinel step (INT_MAX: none)
    PanelCache pc;
    PanelBufs pb;
    // panel block shape per mode (index 0: 1xTF32, 1: 3xTF32, 2: two-float):
    // consumer warps (16-shot groups per task) and ring stages; sfm_autotune
    // overwrites them
    int pncw[3] = {4, 4, 4}, pnstage[3] = {4, 4, 2};
    int* d_task_ptr = nullptr;
    int4* d_task = nullptr;
    int task_grid = -1, task_ncw = -1, task_ngroups = -1;
    Cache<float> c32;
    Cache<double> c64;
    Cache<float2> c2;
    Cache<float> c32f;                 // factored FP32 coefficients
    Cache<float2> c2f;                 // factored FP32 coefficients, two-float state
    RunBufs<float> r32;
    RunBufs<double> r64;
    RunBufs<float2> r2;
    double* d_traces = nullptr;
    size_t n_traces = 0;
    int* d_bad = nullptr;
    unsigned long long timeout_ns = 2000000000ull;
    int skip_arrive = -1;
    // stepping block shape per precision (FP64, FP32, FP32x2, FP32F): consumer
    // warps and coefficient ring stages; sfm_autotune overwrites these
    int ncw[8] = {8, 8, 8, 8, 8, 8, 8, 8}, nstage[8] = {4, 4, 4, 4, 4, 4, 4, 4};
    int* d_piece_ptr = nullptr;
    int4* d_prec = nullptr;            // piece records (sfm::piece_records)
    int piece_grid = -1, piece_units = -1, piece_src = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // state left by the last sfm_run (for sfm_checkpoint): its precision
    // (-1: none), time steps and shot count
    int ck_prec = -1, ck_steps = 0, ck_nshots = 0;
};

static sfm_ext* ext(sfm_handle* h) { return reinterpret_cast<sfm_ext*>(h->scratch); }

static void invalidate(sfm_handle* h) {
    ext(h)->pc.release();
    ext(h)->task_grid = -1;
    ext(h)->c32.release();
    ext(h)->c64.release();
    ext(h)->c2.release();
    ext(h)->c32f.release();
    ext(h)->c2f.release();
}

extern "C" {

int sfm_create(sfm_handle** out, int device) {
    if (!out) return fail(nullptr, SFM_ERR_ARG, "sfm_create: NULL handle pointer");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(nullptr, SFM_ERR_ARG, "sfm_create: bad device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    sfm_handle* h = new (std::nothrow) sfm_handle();
    if (!h) return fail(nullptr, SFM_ERR_NOMEM, "sfm_create: host allocation");
    h->device = device;
    h->scratch = new (std::nothrow) sfm_ext();
    if (!h->scratch) { delete h; return fail(nullptr, SFM_ERR_NOMEM, "sfm_create: host allocation"); }
    sfm_ext* x = ext(h);
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&x->ev0)) != cudaSuccess ||
        (e = cudaEventCreate(&x->ev1)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->d_bar, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void**)&x->d_bad, sizeof(int))) != cudaSuccess) {
        int rc = cuda_fail(nullptr, e, "sfm_create");
        sfm_destroy(h);
        return rc;
    }
    *out = h;
    return SFM_OK;
}

int sfm_destroy(sfm_handle* h) {
    if (!h) return SFM_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    sfm_ext* x = ext(h);
    if (x) {
        x->c32.release(); x->c64.release(); x->c2.release(); x->c32f.release(); x->c2f.release();
        x->r32.release(); x->r64.release(); x->r2.release();
        x->pc.release(); x->pb.release();
        dfree(x->d_ustep);
        dfree(x->d_task_ptr); dfree(x->d_task);
        dfree(x->d_traces); dfree(x->d_bad); dfree(x->d_piece_ptr); dfree(x->d_prec);
        if (x->ev0) cudaEventDestroy(x->ev0);
        if (x->ev1) cudaEventDestroy(x->ev1);
        delete x;
    }
    sfm::free_build(h);
    dfree(h->d_b); dfree(h->d_k); dfree(h->d_face_off); dfree(h->d_nbr);
    dfree(h->d_coef_off); dfree(h->d_H_off); dfree(h->d_state_off); dfree(h->d_mail_off);
    dfree(h->d_tcoef_off);
    dfree(h->d_coef64); dfree(h->d_H64); dfree(h->d_src64); dfree(h->d_src_off);
    dfree(h->d_rrows64); dfree(h->d_rp_sub); dfree(h->d_rec_ptr); dfree(h->d_rec_pairs);
    dfree(h->d_frow); dfree(h->d_rtab); dfree(h->d_init_U64); dfree(h->d_init_V64);
    dfree(h->d_rp_off); dfree(h->d_bar); dfree(h->d_err);
    if (h->stream && h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return SFM_OK;
}

const char* sfm_last_error(const sfm_handle* h) {
    return h ? h->err.c_str() : g_err.c_str();
}

int sfm_set_stream(sfm_handle* h, void* stream) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "sfm_set_stream: NULL handle");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
    h->own_stream = false;
    if (stream) {
        h->stream = (cudaStream_t)stream;      // the caller's: never destroyed here
    } else {
        CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    return SFM_OK;
}

int sfm_set_topology(sfm_handle* h, int nsub, const int* k_sub, const int* m_face,
                     const int* nbr) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (nsub <= 0 || !k_sub || !m_face || !nbr)
        return fail(h, SFM_ERR_ARG, "sfm_set_topology: bad arguments");
    CK(h, cudaSetDevice(h->device));
    ext(h)->piece_grid = -1;   // the per-block pieces follow k_sub
    for (int s = 0; s < nsub; ++s) {
        if (k_sub[s] < 1) return fail(h, SFM_ERR_ARG, "sfm_set_topology: k < 1");
        int b = 0;
        for (int f = 0; f < 6; ++f) {
            const int m = m_face[s * 6 + f], t = nbr[s * 6 + f];
            if (m < 0 || m > SFM_MAX_FACE_M)
                return fail(h, SFM_ERR_ARG, "sfm_set_topology: face mode count out of range");
            if (t >= nsub || t < -1 || t == s)
                return fail(h, SFM_ERR_ARG, "sfm_set_topology: bad neighbour index");
            if (t >= 0 && (nbr[t * 6 + (f ^ 1)] != s || m_face[t * 6 + (f ^ 1)] != m))
                return fail(h, SFM_ERR_ARG, "sfm_set_topology: neighbours not symmetric");
            b += m;
        }
        if (b == 0) return fail(h, SFM_ERR_ARG, "sfm_set_topology: subdomain with b = 0");
        if ((long long)b * k_sub[s] > 256 * 64)
            return fail(h, SFM_ERR_ARG, "sfm_set_topology: k*b too large");
        if (b > sfm::BMAX_WIDE)
            return fail(h, SFM_ERR_ARG, "sfm_set_topology: block width b above " + std::to_string(sfm::BMAX_WIDE));
    }
    h->nsub = nsub;
    h->k.assign(k_sub, k_sub + nsub);
    h->mface.assign(m_face, m_face + 6 * nsub);
    h->nbr.assign(nbr, nbr + 6 * nsub);
    h->b.assign(nsub, 0);
    h->face_off.assign(7 * nsub, 0);
    h->coef_off.assign(nsub, 0);
    h->H_off.assign(6 * nsub, -1);
    h->state_off.assign(nsub, 0);
    h->mail_off.assign(nsub, 0);
    h->tcoef_off.assign(nsub, 0);
    long long co = 0, ho = 0, so = 0, mo = 0, to = 0;
    h->kmax = h->bmax = 0;
    for (int s = 0; s < nsub; ++s) {
        int b = 0;
        for (int f = 0; f < 6; ++f) {
            h->face_off[s * 7 + f] = b;
            const int m = m_face[s * 6 + f];
            if (m > 0) { h->H_off[s * 6 + f] = ho; ho += (long long)m * m; }
            b += m;
        }
        h->face_off[s * 7 + 6] = b;
        h->b[s] = b;
        h->coef_off[s] = co;
        co += 2LL * h->k[s] * b * b;
        h->tcoef_off[s] = to;
        to += 2LL * h->k[s] * sfm::sym_tiles(b) * 64;
        h->state_off[s] = so;
        so += (long long)h->k[s] * b;
        h->mail_off[s] = mo;
        mo += b;
        h->kmax = std::max(h->kmax, h->k[s]);
        h->bmax = std::max(h->bmax, b);
    }
    h->ncoef = co; h->nH = ho; h->nstate = so; h->nmail = mo; h->ntcoef = to;
    cudaStream_t st = h->stream;
    CK(h, upload(h->d_b, h->b.data(), nsub, st));
    CK(h, upload(h->d_k, h->k.data(), nsub, st));
    CK(h, upload(h->d_face_off, h->face_off.data(), 7 * (size_t)nsub, st));
    CK(h, upload(h->d_nbr, h->nbr.data(), 6 * (size_t)nsub, st));
    CK(h, upload(h->d_coef_off, h->coef_off.data(), nsub, st));
    CK(h, upload(h->d_tcoef_off, h->tcoef_off.data(), nsub, st));
    CK(h, upload(h->d_H_off, h->H_off.data(), 6 * (size_t)nsub, st));
    CK(h, upload(h->d_state_off, h->state_off.data(), nsub, st));
    CK(h, upload(h->d_mail_off, h->mail_off.data(), nsub, st));
    {
        std::vector<int4> rows;
        if (!sfm::face_rows(nsub, h->b.data(), h->face_off.data(), h->nbr.data(), h->H_off.data(),
                            h->mail_off.data(), rows))
            return fail(h, SFM_ERR_ARG, "sfm_set_topology: offsets beyond 32 bits");
        CK(h, upload(h->d_frow, rows.data(), rows.size(), st));
    }
    h->have_coef = h->have_src = h->have_rec = h->have_init = false;
    ext(h)->ck_prec = -1;
    invalidate(h);
    return SFM_OK;
}

}  // extern "C"

static int set_coeffs_common(sfm_handle* h, const double* coeffs, bool on_device) {
    CK(h, cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    if (on_device) {
        CK(h, dalloc(h->d_coef64, (size_t)h->ncoef));
        CK(h, cudaMemcpyAsync(h->d_coef64, coeffs, (size_t)h->ncoef * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    } else {
        CK(h, upload(h->d_coef64, coeffs, (size_t)h->ncoef, st));
    }
    CK(h, dalloc(h->d_H64, (size_t)h->nH));
    std::vector<long long> gh1(h->nsub);
    for (int s = 0; s < h->nsub; ++s)
        gh1[s] = h->coef_off[s] + (long long)h->k[s] * h->b[s] * h->b[s];
    long long* d_gh1 = nullptr;
    cudaError_t e = upload(d_gh1, gh1.data(), gh1.size(), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = sfm::launch_face_H(h->d_coef64, d_gh1, h->d_b, h->d_face_off, h->d_nbr, h->d_H_off,
                               h->d_H64, h->nsub, h->d_err, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d_gh1);
    if (e != cudaSuccess) return cuda_fail(h, e, "face coupling H_f");
    invalidate(h);
    if (herr != 0) {
        h->have_coef = false;
        return fail(h, herr, "sfm_set_coeffs: a face block of Gammahat_1 is not SPD");
    }
    h->have_coef = true;
    return SFM_OK;
}

namespace sfm {
int set_topology_internal(sfm_handle* h, int nsub, const int* k_sub, const int* m_face,
                          const int* nbr) {
    return sfm_set_topology(h, nsub, k_sub, m_face, nbr);
}
int set_coeffs_device(sfm_handle* h, const double* d_coeffs) {
    return set_coeffs_common(h, d_coeffs, true);
}
}  // namespace sfm

extern "C" {

int sfm_set_coeffs(sfm_handle* h, const double* coeffs, size_t count) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (h->nsub == 0) return fail(h, SFM_ERR_STATE, "sfm_set_coeffs: no topology");
    if (!coeffs || count != (size_t)h->ncoef)
        return fail(h, SFM_ERR_ARG, "sfm_set_coeffs: count does not match the topology");
    return set_coeffs_common(h, coeffs, false);
}

int sfm_get_coeffs(sfm_handle* h, double* coeffs, size_t count, size_t* needed) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (needed) *needed = (size_t)h->ncoef;
    if (!coeffs) return SFM_OK;
    if (!h->have_coef) return fail(h, SFM_ERR_STATE, "sfm_get_coeffs: no coefficients");
    if (count < (size_t)h->ncoef) return fail(h, SFM_ERR_ARG, "sfm_get_coeffs: buffer too small");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaMemcpyAsync(coeffs, h->d_coef64, h->ncoef * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return SFM_OK;
}

int sfm_set_sources(sfm_handle* h, int nshots, int npairs, const int* pair_shot,
                    const int* pair_sub, const double* rows) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (h->nsub == 0) return fail(h, SFM_ERR_STATE, "sfm_set_sources: no topology");
    if (nshots < 1 || npairs < 0 || (npairs > 0 && (!pair_shot || !pair_sub || !rows)))
        return fail(h, SFM_ERR_ARG, "sfm_set_sources: bad arguments");
    CK(h, cudaSetDevice(h->device));
    std::vector<long long> off((size_t)nshots * h->nsub, -1);
    long long o = 0;
    for (int i = 0; i < npairs; ++i) {
        const int q = pair_shot[i], s = pair_sub[i];
        if (q < 0 || q >= nshots || s < 0 || s >= h->nsub)
            return fail(h, SFM_ERR_ARG, "sfm_set_sources: pair index out of range");
        if (off[(size_t)q * h->nsub + s] >= 0)
            return fail(h, SFM_ERR_ARG, "sfm_set_sources: duplicate (shot, subdomain) pair");
        off[(size_t)q * h->nsub + s] = o;
        o += (long long)h->k[s] * h->b[s];
    }
    h->nshots = nshots;
    h->src_off = off;
    h->nsrc = o;
    CK(h, upload(h->d_src64, rows, (size_t)o, h->stream));
    CK(h, upload(h->d_src_off, off.data(), off.size(), h->stream));
    h->have_src = true;
    ext(h)->piece_grid = -1;   // piece records carry the source offsets
    invalidate(h);
    return SFM_OK;
}

int sfm_set_initial(sfm_handle* h, int nshots, int npairs, const int* pair_shot,
                    const int* pair_sub, const double* u0_rows, const double* v0_rows) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (h->nsub == 0) return fail(h, SFM_ERR_STATE, "sfm_set_initial: no topology");
    if (nshots < 0 || npairs < 0 || (npairs > 0 && (!pair_shot || !pair_sub || !u0_rows)))
        return fail(h, SFM_ERR_ARG, "sfm_set_initial: bad arguments");
    CK(h, cudaSetDevice(h->device));
    if (npairs == 0) {
        h->have_init = false;
        return SFM_OK;
    }
    std::vector<double> U((size_t)nshots * h->nstate, 0.0), V;
    if (v0_rows) V.assign(U.size(), 0.0);
    std::vector<char> seen((size_t)nshots * h->nsub, 0);
    long long o = 0;
    for (int i = 0; i < npairs; ++i) {
        const int q = pair_shot[i], s = pair_sub[i];
        if (q < 0 || q >= nshots || s < 0 || s >= h->nsub)
            return fail(h, SFM_ERR_ARG, "sfm_set_initial: pair index out of range");
        if (seen[(size_t)q * h->nsub + s]++)
            return fail(h, SFM_ERR_ARG, "sfm_set_initial: duplicate (shot, subdomain) pair");
        const long long kb = (long long)h->k[s] * h->b[s];
        const size_t at = (size_t)q * h->nstate + h->state_off[s];
        std::copy(u0_rows + o, u0_rows + o + kb, U.begin() + at);
        if (v0_rows) std::copy(v0_rows + o, v0_rows + o + kb, V.begin() + at);
        o += kb;
    }
    CK(h, upload(h->d_init_U64, U.data(), U.size(), h->stream));
    if (v0_rows) {
        CK(h, upload(h->d_init_V64, V.data(), V.size(), h->stream));
    } else {
        dfree(h->d_init_V64);
    }
    h->init_nshots = nshots;
    h->have_init = true;
    h->init_delta = false;
    return SFM_OK;
}

int sfm_set_receivers(sfm_handle* h, int nrec, int npairs, const int* pair_rec,
                      const int* pair_sub, const double* rows) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (h->nsub == 0) return fail(h, SFM_ERR_STATE, "sfm_set_receivers: no topology");
    if (nrec < 1 || npairs < 0 || (npairs > 0 && (!pair_rec || !pair_sub || !rows)))
        return fail(h, SFM_ERR_ARG, "sfm_set_receivers: bad arguments");
    CK(h, cudaSetDevice(h->device));
    std::vector<int> rsub(npairs), rrec(npairs);
    std::vector<long long> roff(npairs);
    std::vector<int> cnt(nrec + 1, 0);
    long long o = 0;
    for (int i = 0; i < npairs; ++i) {
        const int r = pair_rec[i], s = pair_sub[i];
        if (r < 0 || r >= nrec || s < 0 || s >= h->nsub)
            return fail(h, SFM_ERR_ARG, "sfm_set_receivers: pair index out of range");
        rsub[i] = s; rrec[i] = r; roff[i] = o;
        o += (long long)h->k[s] * h->b[s];
        cnt[r + 1]++;
    }
    for (int r = 0; r < nrec; ++r) cnt[r + 1] += cnt[r];
    std::vector<int> pairs(npairs), fill(cnt.begin(), cnt.end() - 1);
    for (int i = 0; i < npairs; ++i) pairs[fill[rrec[i]]++] = i;
    h->nrec = nrec; h->nrpairs = npairs;
    h->rp_sub = rsub; h->rp_rec = rrec; h->rp_off = roff; h->nrrow = o;
    cudaStream_t st = h->stream;
    CK(h, upload(h->d_rrows64, rows, (size_t)o, st));
    CK(h, upload(h->d_rp_sub, rsub.data(), rsub.size(), st));
    CK(h, upload(h->d_rp_off, roff.data(), roff.size(), st));
    {
        std::vector<int4> tab;
        if (!sfm::readout_table((int)rsub.size(), rsub.data(), roff.data(), h->k.data(), h->b.data(),
                                h->state_off.data(), tab))
            return fail(h, SFM_ERR_ARG, "sfm_set_receivers: offsets beyond 32 bits");
        CK(h, upload(h->d_rtab, tab.data(), tab.size(), st));
    }
    CK(h, upload(h->d_rec_ptr, cnt.data(), cnt.size(), st));
    CK(h, upload(h->d_rec_pairs, pairs.data(), pairs.size(), st));
    h->have_rec = true;
    invalidate(h);
    return SFM_OK;
}

int sfm_debug_set(sfm_handle* h, int key, long long value) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (key == 1) { ext(h)->timeout_ns = (unsigned long long)value; return SFM_OK; }
    if (key == 2) { ext(h)->skip_arrive = (int)value; return SFM_OK; }
    if (key == 3) {
        if (value < 1 || value > 8) return fail(h, SFM_ERR_ARG, "sfm_debug_set: consumer warps 1..8");
        for (int i = 0; i < 8; ++i) ext(h)->ncw[i] = (int)value;
        for (int i = 0; i < 3; ++i) ext(h)->pncw[i] = (int)value;
        return SFM_OK;
    }
    if (key == 4) {
        if (value < 2 || value > 16) return fail(h, SFM_ERR_ARG, "sfm_debug_set: ring stages 2..16");
        for (int i = 0; i < 8; ++i) ext(h)->nstage[i] = (int)value;
        for (int i = 0; i < 3; ++i) ext(h)->pnstage[i] = (int)value;
        return SFM_OK;
    }
    return fail(h, SFM_ERR_ARG, "sfm_debug_set: unknown key");
}

int sfm_plan_pieces(int nunits, int nsub, const int* k_sub, int grid, int* ptr, int* pieces,
                    int max_pieces, int* npieces) {
    if (nunits < 1 || nsub < 1 || nunits % nsub != 0 || !k_sub || grid < 1 || !ptr || !npieces ||
        max_pieces < 0 || (max_pieces > 0 && !pieces))
        return fail(nullptr, SFM_ERR_ARG, "sfm_plan_pieces: bad arguments");
    for (int s = 0; s < nsub; ++s)
        if (k_sub[s] < 1) return fail(nullptr, SFM_ERR_ARG, "sfm_plan_pieces: k < 1");
    std::vector<int> p;
    std::vector<int4> pc;
    sfm::build_pieces(nunits, nsub, k_sub, grid, p, pc);
    *npieces = (int)pc.size();
    std::copy(p.begin(), p.end(), ptr);
    if ((int)pc.size() > max_pieces) return fail(nullptr, SFM_ERR_ARG, "sfm_plan_pieces: max_pieces too small");
    for (size_t i = 0; i < pc.size(); ++i) {
        pieces[3 * i] = pc[i].x;
        pieces[3 * i + 1] = pc[i].y;
        pieces[3 * i + 2] = pc[i].z;
    }
    return SFM_OK;
}

int sfm_last_launches(const sfm_handle* h, int* launches) {
    if (!h || !launches) return SFM_ERR_ARG;
    *launches = h->last_launches;
    return SFM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------

static Cache<double>& cache_of(sfm_handle* h, sfm::PolF64) { return ext(h)->c64; }
static Cache<float>& cache_of(sfm_handle* h, sfm::PolF32) { return ext(h)->c32; }
static Cache<float2>& cache_of(sfm_handle* h, sfm::PolF32x2) { return ext(h)->c2; }
static Cache<float>& cache_of(sfm_handle* h, sfm::PolF32F) { return ext(h)->c32f; }
static Cache<float2>& cache_of(sfm_handle* h, sfm::PolF32Fx2) { return ext(h)->c2f; }
template <typename T>
static RunBufs<T>& bufs_of(sfm_handle* h);
template <>
RunBufs<float>& bufs_of<float>(sfm_handle* h) { return ext(h)->r32; }
template <>
RunBufs<double>& bufs_of<double>(sfm_handle* h) { return ext(h)->r64; }
template <>
RunBufs<float2>& bufs_of<float2>(sfm_handle* h) { return ext(h)->r2; }

template <class P>
static int prepare(sfm_handle* h) {
    using T = typename P::S;
    auto& c = cache_of(h, P{});
    if (c.valid) return SFM_OK;
    c.release();
    cudaStream_t st = h->stream;
    if constexpr (P::factored) CK(h, dalloc(c.fcoef, (size_t)h->ntcoef));
    else CK(h, dalloc(c.coef, (size_t)h->ntcoef));
    CK(h, dalloc(c.H, (size_t)h->nH));
    CK(h, dalloc(c.src, (size_t)h->nsrc));
    CK(h, dalloc(c.rrows, (size_t)h->nrrow));
    int bad = 0;
    if constexpr (P::factored) {
        CK(h, cudaMemsetAsync(ext(h)->d_bad, 0, sizeof(int), st));
        CK(h, sfm::launch_factor_tiles(h->d_coef64, h->d_coef_off, h->d_tcoef_off, h->d_b, h->d_k,
                                       h->nsub, h->kmax, c.fcoef, ext(h)->d_bad, st));
        CK(h, cudaMemcpyAsync(&bad, ext(h)->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    } else {
        CK(h, sfm::launch_pack_tiles<P>(h->d_coef64, h->d_coef_off, h->d_tcoef_off, h->d_b, h->d_k,
                                        h->nsub, c.coef, st));
    }
    CK(h, sfm::launch_convert<P>(h->d_H64, c.H, (size_t)h->nH, st));
    CK(h, sfm::launch_convert<P>(h->d_src64, c.src, (size_t)h->nsrc, st));
    CK(h, sfm::launch_convert<P>(h->d_rrows64, c.rrows, (size_t)h->nrrow, st));
    CK(h, cudaStreamSynchronize(st));
    if (bad) {
        c.release();
        return fail(h, SFM_ERR_NOT_SPD, "factored FP32: an S-fraction block is not positive definite");
    }
    c.valid = true;
    return SFM_OK;
}

static int prec_id(sfm::PolF64) { return SFM_FP64; }
static int prec_id(sfm::PolF32) { return SFM_FP32; }
static int prec_id(sfm::PolF32x2) { return SFM_FP32X2; }
static int prec_id(sfm::PolF32F) { return SFM_FP32F; }
static int prec_id(sfm::PolF32Fx2) { return SFM_FP32FX2; }

// Grid of the persistent stepping kernel (co-resident blocks for the
// chosen shape, at most one per level of work) and the per-block pieces.
// src_off: host source offsets per (shot, subdomain), NULL for none (kind 0).
template <class P>
static int step_setup(sfm_handle* h, int nunits, const long long* src_off,
                      sfm::StepParams<typename P::S>& p, int* grid_out) {
    sfm_ext* x = ext(h);
    const int id = prec_id(P{});
    // a policy's kernel may take fewer consumer warps than asked for
    const int ncw = std::min(x->ncw[id], sfm::step_max_ncw<P>());
    int nstage = x->nstage[id];
    // factored blocks are owned by warp (block index mod ncw) through fixed
    // stages: the ring depth must be a multiple of the warp count
    if (P::factored) nstage = (nstage + ncw - 1) / ncw * ncw;
    // wide blocks: fewer ring stages when the requested ring does not fit
    {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int step = P::factored ? ncw : 1;
        while (nstage - step >= 2 && sfm::step_smem_bytes<P>(h->kmax, h->bmax, nstage) > (size_t)optin)
            nstage -= step;
    }
    int gmax = 0;
    if (sfm::step_max_grid<P>(ncw, sfm::step_smem_bytes<P>(h->kmax, h->bmax, nstage), &gmax) != 0)
        return fail(h, SFM_ERR_ARG, "stepping: subdomain blocks too large for shared memory");
    long long levels = 0;
    for (int u = 0; u < nunits; ++u) levels += h->k[u % h->nsub];
    const int grid = (int)std::max(1LL, std::min<long long>(gmax, levels));
    const int src_kind = src_off ? 1 : 0;
    if (grid != x->piece_grid || nunits != x->piece_units || src_kind != x->piece_src) {
        std::vector<int> ptr;
        std::vector<int4> pieces, rec;
        sfm::build_pieces(nunits, h->nsub, h->k.data(), grid, ptr, pieces);
        std::vector<long long> none;
        if (!src_off) { none.assign((size_t)nunits, -1); src_off = none.data(); }
        if (!sfm::piece_records(pieces, h->nsub, h->k.data(), h->b.data(), h->state_off.data(),
                                src_off, h->mail_off.data(), rec))
            return fail(h, SFM_ERR_ARG, "stepping: offsets beyond 32 bits");
        CK(h, upload(x->d_piece_ptr, ptr.data(), ptr.size(), h->stream));
        CK(h, upload(x->d_prec, rec.data(), rec.size(), h->stream));
        x->piece_grid = grid;
        x->piece_units = nunits;
        x->piece_src = src_kind;
    }
    p.ncw = ncw;
    p.nstage = nstage;
    p.stage_v4 = 0;
    if (P::factored) {
        // 16-byte staging copies when every width is a whole number of them
        const int epv = (int)(16 / sizeof(typename P::S));
        p.stage_v4 = 1;
        for (int s = 0; s < h->nsub; ++s)
            if (h->b[s] % epv != 0) p.stage_v4 = 0;
    }
    p.piece_ptr = x->d_piece_ptr;
    p.prec = x->d_prec;
    p.frow = h->d_frow;
    *grid_out = grid;
    return SFM_OK;
}

template <typename P>
static cudaError_t grow(P*& p, size_t& have, size_t need) {
    if (need <= have && p) return cudaSuccess;
    cudaError_t e = dalloc(p, need);
    have = (e == cudaSuccess) ? need : 0;
    return e;
}

// Right-hand side without the source for every shot of the initial state:
// one step of the FP64 stepping kernel from state X (state layout, all
// shots) with zero increment, zero source and dt = 1 leaves a_hom(X) in the
// increment buffer A.
static int accel_f64(sfm_handle* h, const double* X, double* A, int* launches) {
    int rc = prepare<sfm::PolF64>(h);
    if (rc != SFM_OK) return rc;
    sfm_ext* x = ext(h);
    Cache<double>& c = x->c64;
    cudaStream_t st = h->stream;
    const int nsh = h->init_nshots;
    const size_t n = (size_t)nsh * h->nstate;
    double *U0 = nullptr, *U1 = nullptr, *m0 = nullptr, *m1 = nullptr, *wav = nullptr;
    unsigned* ctr = nullptr;
    auto cleanup = [&]() { dfree(U0); dfree(U1); dfree(m0); dfree(m1); dfree(wav); dfree(ctr); };
#define CKA(call)                                                              \
    do {                                                                       \
        cudaError_t e__ = (call);                                              \
        if (e__ != cudaSuccess) { cleanup(); return cuda_fail(h, e__, #call); } \
    } while (0)
    CKA(dalloc(U0, n));
    CKA(dalloc(U1, n));
    CKA(dalloc(m0, (size_t)nsh * h->nmail));
    CKA(dalloc(m1, (size_t)nsh * h->nmail));
    CKA(dalloc(wav, (size_t)nsh));
    CKA(dalloc(ctr, 2));
    CKA(cudaMemcpyAsync(U0, X, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CKA(cudaMemsetAsync(A, 0, n * sizeof(double), st));
    CKA(cudaMemsetAsync(wav, 0, (size_t)nsh * sizeof(double), st));
    CKA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), st));
    CKA(cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), st));
    CKA(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    sfm::StepParams<double> p{};
    p.nsub = h->nsub; p.nshots = nsh; p.nunits = nsh * h->nsub; p.nsteps = 1;
    p.kmax = h->kmax; p.bmax = h->bmax;
    p.sub_b = h->d_b; p.sub_k = h->d_k; p.coef_off = h->d_tcoef_off; p.coef = c.coef;
    p.face_off = h->d_face_off; p.nbr = h->d_nbr; p.H_off = h->d_H_off; p.H = c.H;
    p.state_off = h->d_state_off; p.state_stride = h->nstate;
    p.U[0] = U0; p.U[1] = U1; p.U[2] = p.U[3] = nullptr;
    p.dU = A;
    p.mail_off = h->d_mail_off; p.mail_stride = h->nmail; p.mail0 = m0; p.mail1 = m1;
    p.src_off = nullptr; p.src = c.src; p.wavelet = wav;
    p.nrec = 0; p.nrpairs = 0; p.rp_sub = nullptr; p.rp_off = nullptr; p.rrows = nullptr;
    p.partial = nullptr; p.rctr = ctr;
    p.dt2 = 1.0;
    p.bar = h->d_bar; p.err = h->d_err; p.timeout_ns = x->timeout_ns; p.skip_arrive = -1;
    p.Kx = nullptr;
    int grid = 0;
    rc = step_setup<sfm::PolF64>(h, p.nunits, nullptr, p, &grid);
    if (rc != SFM_OK) { cleanup(); return rc; }
    p.rtab = nullptr;
    CKA(sfm::launch_step<sfm::PolF64>(p, grid, st));
    ++*launches;
    int herr = 0;
    CKA(cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKA(cudaStreamSynchronize(st));
#undef CKA
    cleanup();
    if (herr != 0) return fail(h, herr, "initial state: device error");
    return SFM_OK;
}

// Discrete energy E = 1/2 (delta/dt)^T MM (delta/dt) + 1/2 U^T KK (U - delta)
// per shot of a state (U, delta) in the state layout (energy.cu), in FP64;
// the per-(subdomain, level) terms are added on the host in a fixed order.
static int energy_f64(sfm_handle* h, const double* U, const double* D, int nshots, double dt,
                      double* out) {
    cudaStream_t st = h->stream;
    const size_t nt = (size_t)nshots * h->nsub * h->kmax * 2;
    double* d_t = nullptr;
    CK(h, dalloc(d_t, nt));
    std::vector<double> t(nt);
    cudaError_t e = sfm::launch_energy_terms(h->d_coef64, h->d_coef_off, h->d_b, h->d_k, h->nsub,
                                             h->kmax, nshots, U, D, h->nstate, h->d_state_off, d_t, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.data(), d_t, nt * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d_t);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy");
    for (int q = 0; q < nshots; ++q) {
        double kin = 0.0, pot = 0.0;
        for (int s = 0; s < h->nsub; ++s)
            for (int j = 0; j < h->k[s]; ++j) {
                const size_t i = (((size_t)q * h->nsub + s) * h->kmax + j) * 2;
                kin += t[i];
                pot += t[i + 1];
            }
        out[q] = 0.5 * kin / (dt * dt) + 0.5 * pot;
    }
    return SFM_OK;
}

template <typename T>
static int energy_of(sfm_handle* h, const T* U, const T* D, int nshots, double dt, double* out) {
    if constexpr (std::is_same<T, double>::value) {
        return energy_f64(h, U, D, nshots, dt, out);
    } else {
        const size_t n = (size_t)nshots * h->nstate;
        double *U64 = nullptr, *D64 = nullptr;
        cudaError_t e = dalloc(U64, n);
        if (e == cudaSuccess) e = dalloc(D64, n);
        if (e == cudaSuccess) e = sfm::launch_state_to_f64<T>(U, U64, n, h->stream);
        if (e == cudaSuccess) e = sfm::launch_state_to_f64<T>(D, D64, n, h->stream);
        int rc = e == cudaSuccess ? energy_f64(h, U64, D64, nshots, dt, out) : cuda_fail(h, e, "energy");
        dfree(U64);
        dfree(D64);
        return rc;
    }
}

// panel state (FP32 panels, or two-float panels in mode 2) -> FP64 state layout
static cudaError_t from_panel_any(int mode, const float* in, double* out, int nshots, long long n,
                                  cudaStream_t st) {
    return mode == 2 ? sfm::launch_from_panel2(in, out, nshots, n, st)
                     : sfm::launch_from_panel(in, out, nshots, n, st);
}

static cudaError_t to_panel_any(int mode, const double* in, float* out, int nshots, long long n,
                                cudaStream_t st) {
    return mode == 2 ? sfm::launch_to_panel2(in, out, nshots, n, st) : sfm::launch_to_panel(in, out, nshots, n, st);
}

static int energy_of_panel(sfm_handle* h, int mode, const float* U, const float* D, int nshots, double dt,
                           double* out) {
    const size_t n = (size_t)nshots * h->nstate;
    double *U64 = nullptr, *D64 = nullptr;
    cudaError_t e = dalloc(U64, n);
    if (e == cudaSuccess) e = dalloc(D64, n);
    if (e == cudaSuccess) e = from_panel_any(mode, U, U64, nshots, h->nstate, h->stream);
    if (e == cudaSuccess) e = from_panel_any(mode, D, D64, nshots, h->nstate, h->stream);
    int rc = e == cudaSuccess ? energy_f64(h, U64, D64, nshots, dt, out) : cuda_fail(h, e, "energy");
    dfree(U64);
    dfree(D64);
    return rc;
}

static int ensure_ustep(sfm_handle* h) {
    sfm_ext* x = ext(h);
    if (!x->d_ustep) CK(h, dalloc(x->d_ustep, 1));
    const int big = INT_MAX;
    CK(h, cudaMemcpyAsync(x->d_ustep, &big, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    return SFM_OK;
}

template <class P>
static int run_impl(sfm_handle* h, double dt, int nsteps, const double* wavelet, double* traces,
                    int flags, double* kernel_ms) {
    using T = typename P::S;
    sfm_ext* x = ext(h);
    if (P::factored && h->bmax > sfm::BMAX_NARROW)
        return fail(h, SFM_ERR_ARG, "factored modes: blocks wider than 64 (a factor product is one "
                                    "warp's registers); use SFM_FP64, SFM_FP32X2 or SFM_FP32");
    int rc = prepare<P>(h);
    if (rc != SFM_OK) return rc;
    auto& c = cache_of(h, P{});
    RunBufs<T>& r = bufs_of<T>(h);
    cudaStream_t st = h->stream;
    const size_t nst = (size_t)h->nshots * h->nstate;
    const size_t nml = (size_t)h->nshots * h->nmail;
    const size_t nwav = (size_t)h->nshots * nsteps;
    const size_t npart = (size_t)h->nshots * (nsteps + 1) * h->nrpairs;
    const size_t ntr = (size_t)h->nshots * h->nrec * (nsteps + 1);
    size_t have_state = r.n_state;
    for (int i = 0; i < 4; ++i) { size_t hs = have_state; CK(h, grow(r.U[i], hs, nst)); }
    { size_t hs = have_state; CK(h, grow(r.dU, hs, nst)); r.n_state = hs; }
    size_t have_mail = r.n_mail;
    { size_t hm = have_mail; CK(h, grow(r.mail[0], hm, nml)); }
    { size_t hm = have_mail; CK(h, grow(r.mail[1], hm, nml)); r.n_mail = hm; }
    CK(h, grow(r.wavelet, r.n_wav, nwav));
    CK(h, grow(r.partial, r.n_part, npart));
    CK(h, grow(r.rctr, r.n_ctr, (size_t)nsteps + 1));
    double* d_traces = traces;
    if (!(flags & SFM_DEVICE_PTR)) {
        CK(h, grow(x->d_traces, x->n_traces, ntr));
        d_traces = x->d_traces;
    }
    // wavelet to the compute precision
    const double* d_wav64 = wavelet;
    double* tmp64 = nullptr;
    if (!(flags & SFM_DEVICE_PTR)) {
        CK(h, dalloc(tmp64, nwav));
        CK(h, cudaMemcpyAsync(tmp64, wavelet, nwav * sizeof(double), cudaMemcpyHostToDevice, st));
        d_wav64 = tmp64;
    }
    int launches = 0;
    CK(h, sfm::launch_convert<P>(d_wav64, r.wavelet, nwav, st));
    ++launches;
    for (int i = 0; i < 4; ++i) CK(h, cudaMemsetAsync(r.U[i], 0, nst * sizeof(T), st));
    CK(h, cudaMemsetAsync(r.rctr, 0, ((size_t)nsteps + 1) * sizeof(unsigned), st));
    CK(h, cudaMemsetAsync(r.dU, 0, nst * sizeof(T), st));
    if (h->have_init && h->init_delta) {
        // state restored by sfm_restore: U^0 and delta^0 themselves
        if (h->init_nshots != h->nshots) {
            dfree(tmp64);
            return fail(h, SFM_ERR_STATE, "sfm_run: restored state has a different shot count");
        }
        cudaError_t e1 = sfm::launch_convert<P>(h->d_init_U64, r.U[0], nst, st);
        if (e1 == cudaSuccess) e1 = sfm::launch_convert<P>(h->d_init_V64, r.dU, nst, st);
        launches += 2;
        if (e1 != cudaSuccess) { dfree(tmp64); return cuda_fail(h, e1, "restored state"); }
    } else if (h->have_init) {
        // Algorithm 1 step 1.4: U^0 given, delta^0 = dt V^0 - dt^2/2 a_hom(U^0)
        // (the second-order Taylor start in increment form), computed in FP64
        if (h->init_nshots != h->nshots) {
            dfree(tmp64);
            return fail(h, SFM_ERR_STATE, "sfm_run: initial state set for a different shot count");
        }
        double *A = nullptr, *D = nullptr;
        cudaError_t e0 = dalloc(A, nst);
        if (e0 == cudaSuccess) e0 = dalloc(D, nst);
        if (e0 != cudaSuccess) { dfree(A); dfree(D); dfree(tmp64); return cuda_fail(h, e0, "initial state"); }
        rc = accel_f64(h, h->d_init_U64, A, &launches);
        cudaError_t e1 = cudaSuccess;
        if (rc == SFM_OK) {
            if ((e1 = sfm::launch_start_delta(h->d_init_V64, A, dt, nst, D, st)) == cudaSuccess &&
                (e1 = sfm::launch_convert<P>(h->d_init_U64, r.U[0], nst, st)) == cudaSuccess &&
                (e1 = sfm::launch_convert<P>(D, r.dU, nst, st)) == cudaSuccess)
                e1 = cudaStreamSynchronize(st);
            launches += 3;
        }
        dfree(A);
        dfree(D);
        if (rc != SFM_OK) { dfree(tmp64); return rc; }
        if (e1 != cudaSuccess) { dfree(tmp64); return cuda_fail(h, e1, "initial state"); }
        CK(h, cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), st));
        CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    }
    CK(h, cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), st));
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    CK(h, cudaMemsetAsync(x->d_bad, 0, sizeof(int), st));
    if (flags & SFM_ENERGY) {
        x->energy.assign(2 * (size_t)h->nshots, 0.0);
        rc = energy_of<T>(h, r.U[0], r.dU, h->nshots, dt, x->energy.data());
        if (rc != SFM_OK) { dfree(tmp64); return rc; }
    }
    rc = ensure_ustep(h);
    if (rc != SFM_OK) { dfree(tmp64); return rc; }

    sfm::StepParams<T> p{};
    p.nsub = h->nsub; p.nshots = h->nshots; p.nunits = h->nshots * h->nsub; p.nsteps = nsteps;
    p.kmax = h->kmax; p.bmax = h->bmax;
    p.sub_b = h->d_b; p.sub_k = h->d_k; p.coef_off = h->d_tcoef_off; p.coef = c.coef;
    p.fcoef = c.fcoef;
    p.face_off = h->d_face_off; p.nbr = h->d_nbr; p.H_off = h->d_H_off; p.H = c.H;
    p.state_off = h->d_state_off; p.state_stride = h->nstate;
    for (int i = 0; i < 4; ++i) p.U[i] = r.U[i];
    p.rctr = r.rctr;
    p.dU = r.dU;
    p.mail_off = h->d_mail_off; p.mail_stride = h->nmail; p.mail0 = r.mail[0]; p.mail1 = r.mail[1];
    p.src_off = h->d_src_off; p.src = c.src; p.wavelet = r.wavelet;
    p.nrec = h->nrec; p.nrpairs = h->nrpairs; p.rp_sub = h->d_rp_sub; p.rp_off = h->d_rp_off;
    p.rrows = c.rrows; p.partial = r.partial;
    p.dt2 = dt * dt;
    p.bar = h->d_bar; p.err = h->d_err; p.timeout_ns = x->timeout_ns;
    p.skip_arrive = x->skip_arrive;
    p.Kx = nullptr;
    p.ustep = x->d_ustep;

    int grid = 0;
    rc = step_setup<P>(h, p.nunits, h->src_off.data(), p, &grid);
    p.rtab = h->d_rtab;
    if (rc != SFM_OK) { dfree(tmp64); return rc; }
    CK(h, cudaEventRecord(x->ev0, st));
    cudaError_t e = sfm::launch_step<P>(p, grid, st);
    if (e != cudaSuccess) { dfree(tmp64); return cuda_fail(h, e, "step kernel launch"); }
    ++launches;
    CK(h, cudaEventRecord(x->ev1, st));
    e = sfm::launch_reduce_traces<P>(r.partial, h->d_rec_ptr, h->d_rec_pairs, h->nshots, nsteps,
                                     h->nrec, h->nrpairs, d_traces, x->d_bad, st);
    if (e != cudaSuccess) { dfree(tmp64); return cuda_fail(h, e, "trace reduction launch"); }
    ++launches;
    int herr = 0, bad = 0;
    CK(h, cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaMemcpyAsync(&bad, x->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!(flags & SFM_DEVICE_PTR))
        CK(h, cudaMemcpyAsync(traces, d_traces, ntr * sizeof(double), cudaMemcpyDeviceToHost, st));
    int ustep = INT_MAX;
    CK(h, cudaMemcpyAsync(&ustep, x->d_ustep, sizeof(int), cudaMemcpyDeviceToHost, st));
    e = cudaStreamSynchronize(st);
    dfree(tmp64);
    if (e != cudaSuccess) return cuda_fail(h, e, "stepping");
    h->last_launches = launches;
    x->info.unstable_step = ustep == INT_MAX ? -1 : ustep;
    if (kernel_ms) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, x->ev0, x->ev1);
        *kernel_ms = ms;
    }
    if (herr == SFM_ERR_TIMEOUT) return fail(h, SFM_ERR_TIMEOUT, "device-wide barrier timed out");
    if (herr == SFM_ERR_UNSTABLE)
        return fail(h, SFM_ERR_UNSTABLE, "unstable: the state ran away at step " +
                                             std::to_string(x->info.unstable_step) +
                                             " (time step above the CFL limit?)");
    if (herr != 0) return fail(h, herr, "device error during stepping");
    if (bad) return fail(h, SFM_ERR_UNSTABLE, "non-finite traces (time step above the CFL limit?)");
    if (flags & SFM_ENERGY) {
        rc = energy_of<T>(h, r.U[nsteps & 3], r.dU, h->nshots, dt, x->energy.data() + h->nshots);
        if (rc != SFM_OK) return rc;
    }
    return SFM_OK;
}

// ---------------------------------------------------------------------------
// Multi-shot panel modes (SFM_TF32X3, SFM_TF32, SFM_FP32X2P): shots stepped
// 16 at a time with tensor-core factor products or two-float CUDA-core
// products (panel.cu).

static bool is_panel(int precision) {
    return precision == SFM_TF32X3 || precision == SFM_TF32 || precision == SFM_FP32X2P;
}
static int panel_mode_of(int precision) {
    return precision == SFM_TF32X3 ? 3 : precision == SFM_FP32X2P ? 2 : 1;
}
static int panel_slot(int mode) { return mode == 3 ? 1 : mode == 2 ? 2 : 0; }

// FP32 data of the panel path, built once per set of coefficients, sources
// and receivers: the FP32 Cholesky factors (factored in FP64) in 72-float
// padded tiles, H_f and the receiver rows in FP32, the source rows of every
// (shot, subdomain) pair in the panel of its (group, subdomain) unit.
static int prepare_panel2(sfm_handle* h);

static int prepare_panel(sfm_handle* h, int mode) {
    sfm_ext* x = ext(h);
    PanelCache& c = x->pc;
    const int ngroups = (h->nshots + 15) / 16;
    if (c.valid && c.ngroups == ngroups) return mode == 2 ? prepare_panel2(h) : SFM_OK;
    c.release();
    cudaStream_t st = h->stream;
    const long long ntiles = h->ntcoef / 64;
    float* tmp = nullptr;
    CK(h, dalloc(tmp, (size_t)h->ntcoef));
    int bad = 0;
    cudaError_t e = cudaMemsetAsync(x->d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = sfm::launch_factor_tiles(h->d_coef64, h->d_coef_off, h->d_tcoef_off, h->d_b, h->d_k,
                                     h->nsub, h->kmax, tmp, x->d_bad, st);
    if (e == cudaSuccess) e = dalloc(c.coef, (size_t)ntiles * 72);
    if (e == cudaSuccess) e = sfm::launch_pad_tiles(tmp, c.coef, ntiles, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, x->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(tmp);
    if (e != cudaSuccess) { c.release(); return cuda_fail(h, e, "panel factors"); }
    if (bad) {
        c.release();
        return fail(h, SFM_ERR_NOT_SPD, "panel modes: an S-fraction block is not positive definite");
    }
    std::vector<long long> coff(h->nsub);
    for (int s = 0; s < h->nsub; ++s) coff[s] = h->tcoef_off[s] / 64 * 72;
    CK(h, upload(c.d_coef_off, coff.data(), coff.size(), st));
    CK(h, dalloc(c.H, (size_t)h->nH));
    CK(h, sfm::launch_convert<sfm::PolF32F>(h->d_H64, c.H, (size_t)h->nH, st));
    CK(h, dalloc(c.rrows, (size_t)h->nrrow));
    CK(h, sfm::launch_convert<sfm::PolF32F>(h->d_rrows64, c.rrows, (size_t)h->nrrow, st));
    // source panels
    std::vector<long long> poff((size_t)ngroups * h->nsub, -1), off64, dst;
    std::vector<int> len;
    long long total = 0;
    for (int q = 0; q < h->nshots; ++q)
        for (int s = 0; s < h->nsub; ++s) {
            const long long so = h->src_off[(size_t)q * h->nsub + s];
            if (so < 0) continue;
            long long& po = poff[(size_t)(q / 16) * h->nsub + s];
            if (po < 0) { po = total; total += (long long)h->k[s] * h->b[s] * 16; }
            const int c16 = q % 16;
            off64.push_back(so);
            dst.push_back(po + 2 * (c16 & 7) + (c16 >> 3));
            len.push_back(h->k[s] * h->b[s]);
        }
    CK(h, upload(c.d_src_off, poff.data(), poff.size(), st));
    CK(h, dalloc(c.src, (size_t)std::max<long long>(total, 1)));
    if (total) CK(h, cudaMemsetAsync(c.src, 0, (size_t)total * sizeof(float), st));
    if (!off64.empty()) {
        long long *d_o = nullptr, *d_d = nullptr;
        int* d_l = nullptr;
        e = upload(d_o, off64.data(), off64.size(), st);
        if (e == cudaSuccess) e = upload(d_d, dst.data(), dst.size(), st);
        if (e == cudaSuccess) e = upload(d_l, len.data(), len.size(), st);
        if (e == cudaSuccess) e = sfm::launch_src_panels(h->d_src64, d_o, d_d, d_l, (int)off64.size(), c.src, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        dfree(d_o); dfree(d_d); dfree(d_l);
        if (e != cudaSuccess) { c.release(); return cuda_fail(h, e, "panel sources"); }
    }
    // receiver pairs by subdomain
    std::vector<int> ptr(h->nsub + 1, 0), list(std::max(h->nrpairs, 1));
    for (int i = 0; i < h->nrpairs; ++i) ptr[h->rp_sub[i] + 1]++;
    for (int s = 0; s < h->nsub; ++s) ptr[s + 1] += ptr[s];
    {
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int i = 0; i < h->nrpairs; ++i) list[fill[h->rp_sub[i]]++] = i;
    }
    int rpmax = 0;
    for (int s = 0; s < h->nsub; ++s) rpmax = std::max(rpmax, ptr[s + 1] - ptr[s]);
    CK(h, upload(c.d_sub_rp_ptr, ptr.data(), ptr.size(), st));
    CK(h, upload(c.d_sub_rp, list.data(), list.size(), st));
    c.ngroups = ngroups;
    c.rpmax = rpmax;
    c.valid = true;
    return mode == 2 ? prepare_panel2(h) : SFM_OK;
}

// Two-float data of SFM_FP32X2P (once per set of coefficients): the
// symmetric blocks in padded two-float tiles, H_f and the receiver rows as
// (hi, lo) pairs.
static int prepare_panel2(sfm_handle* h) {
    PanelCache& c = ext(h)->pc;
    if (c.coef2) return SFM_OK;
    cudaStream_t st = h->stream;
    const long long ntiles = h->ntcoef / 64;
    std::vector<long long> coff(h->nsub);
    for (int s = 0; s < h->nsub; ++s) coff[s] = h->tcoef_off[s] / 64 * 144;
    cudaError_t e = dalloc(c.coef2, (size_t)ntiles * 144);
    if (e == cudaSuccess) e = sfm::launch_pack_sym2(h->d_coef64, h->d_coef_off, h->d_tcoef_off, h->d_b, h->d_k,
                                                    h->nsub, c.coef2, st);
    if (e == cudaSuccess) e = upload(c.d_coef2_off, coff.data(), coff.size(), st);
    if (e == cudaSuccess) e = dalloc(c.H2, 2 * (size_t)h->nH);
    if (e == cudaSuccess)
        e = sfm::launch_convert<sfm::PolF32x2>(h->d_H64, reinterpret_cast<float2*>(c.H2), (size_t)h->nH, st);
    if (e == cudaSuccess) e = dalloc(c.rrows2, 2 * (size_t)std::max<long long>(h->nrrow, 1));
    if (e == cudaSuccess && h->nrrow > 0)
        e = sfm::launch_convert<sfm::PolF32x2>(h->d_rrows64, reinterpret_cast<float2*>(c.rrows2),
                                               (size_t)h->nrrow, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dfree(c.coef2); dfree(c.H2); dfree(c.rrows2); dfree(c.d_coef2_off);
        return cuda_fail(h, e, "two-float panel data");
    }
    return SFM_OK;
}

// Block shape, grid and task table of the panel kernel for this handle.
static int panel_setup(sfm_handle* h, int mode, int* grid_out, int* ncw_out, int* nstage_out) {
    sfm_ext* x = ext(h);
    const int slot = panel_slot(mode);
    const int ngroups = x->pc.ngroups;
    const int ncw = std::max(1, std::min(x->pncw[slot], std::min(ngroups, sfm::panel_max_ncw(mode))));
    const int nstage = x->pnstage[slot];
    const size_t smem = sfm::panel_smem_bytes(mode, ncw, nstage, h->bmax, x->pc.rpmax);
    int gmax = 0;
    if (sfm::panel_max_grid(mode, ncw, smem, &gmax) != 0)
        return fail(h, SFM_ERR_ARG, "panel modes: blocks too large for shared memory");
    const long long ntasks = (long long)h->nsub * ((ngroups + ncw - 1) / ncw);
    const int grid = (int)std::max(1LL, std::min<long long>(gmax, ntasks));
    if (grid != x->task_grid || ncw != x->task_ncw || ngroups != x->task_ngroups) {
        std::vector<int> ptr;
        std::vector<int4> tasks;
        sfm::build_panel_tasks(h->nsub, ngroups, h->k.data(), h->b.data(), ncw, grid, ptr, tasks);
        CK(h, upload(x->d_task_ptr, ptr.data(), ptr.size(), h->stream));
        CK(h, upload(x->d_task, tasks.data(), tasks.size(), h->stream));
        x->task_grid = grid;
        x->task_ncw = ncw;
        x->task_ngroups = ngroups;
    }
    *grid_out = grid;
    *ncw_out = ncw;
    *nstage_out = nstage;
    return SFM_OK;
}

// The panel run: like run_impl, with the state, face data, wavelet and
// readout sums in panel form.  zero_source: a probe with a zero wavelet
// from rest (sfm_autotune), leaving any initial state aside.
static int run_panel_impl(sfm_handle* h, int mode, double dt, int nsteps, const double* wavelet,
                          double* traces, int flags, double* kernel_ms, bool zero_source = false) {
    sfm_ext* x = ext(h);
    if (h->bmax > sfm::BMAX_NARROW)
        return fail(h, SFM_ERR_ARG, "panel modes: blocks wider than 64 (eight 8-row tiles a warp)");
    int rc = prepare_panel(h, mode);
    if (rc != SFM_OK) return rc;
    PanelCache& c = x->pc;
    PanelBufs& r = x->pb;
    cudaStream_t st = h->stream;
    const int ngroups = c.ngroups;
    const size_t words = mode == 2 ? 2 : 1;            // floats per number
    const size_t nst = (size_t)ngroups * h->nstate * 16 * words;
    const size_t nml = (size_t)ngroups * h->nmail * 16 * words;
    const size_t nwav = (size_t)ngroups * 16 * nsteps;
    const size_t npart = (size_t)ngroups * (nsteps + 1) * std::max(h->nrpairs, 1) * 16 * words;
    const size_t ntr = (size_t)h->nshots * h->nrec * (nsteps + 1);
    { size_t hs = r.n_state; CK(h, grow(r.U, hs, nst)); }
    { size_t hs = r.n_state; CK(h, grow(r.dU, hs, nst)); r.n_state = hs; }
    { size_t hm = r.n_mail; CK(h, grow(r.mail[0], hm, nml)); }
    { size_t hm = r.n_mail; CK(h, grow(r.mail[1], hm, nml)); r.n_mail = hm; }
    CK(h, grow(r.wav, r.n_wav, nwav));
    CK(h, grow(r.partial, r.n_part, npart));
    double* d_traces = traces;
    if (!(flags & SFM_DEVICE_PTR)) {
        CK(h, grow(x->d_traces, x->n_traces, ntr));
        d_traces = x->d_traces;
    }
    int launches = 0;
    CK(h, cudaMemsetAsync(r.wav, 0, nwav * sizeof(float), st));
    if (!zero_source) {
        const size_t nw64 = (size_t)h->nshots * nsteps;
        const double* d_wav64 = wavelet;
        double* tmp64 = nullptr;
        if (!(flags & SFM_DEVICE_PTR)) {
            CK(h, dalloc(tmp64, nw64));
            cudaError_t e = cudaMemcpyAsync(tmp64, wavelet, nw64 * sizeof(double), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { dfree(tmp64); return cuda_fail(h, e, "wavelet"); }
            d_wav64 = tmp64;
        }
        cudaError_t e = sfm::launch_convert<sfm::PolF32F>(d_wav64, r.wav, nw64, st);
        if (e == cudaSuccess && tmp64) e = cudaStreamSynchronize(st);
        dfree(tmp64);
        if (e != cudaSuccess) return cuda_fail(h, e, "wavelet");
        ++launches;
    }
    CK(h, cudaMemsetAsync(r.U, 0, nst * sizeof(float), st));
    CK(h, cudaMemsetAsync(r.dU, 0, nst * sizeof(float), st));
    if (h->have_init && !zero_source) {
        if (h->init_nshots != h->nshots)
            return fail(h, SFM_ERR_STATE, "sfm_run: initial state set for a different shot count");
        if (h->init_delta) {
            // restored U^0 and delta^0
            CK(h, to_panel_any(mode, h->d_init_U64, r.U, h->nshots, h->nstate, st));
            CK(h, to_panel_any(mode, h->d_init_V64, r.dU, h->nshots, h->nstate, st));
            launches += 2;
        } else {
            // delta^0 = dt V^0 - dt^2/2 a_hom(U^0), in FP64 (Algorithm 1 step 1.4)
            const size_t n64 = (size_t)h->nshots * h->nstate;
            double *A = nullptr, *D = nullptr;
            cudaError_t e0 = dalloc(A, n64);
            if (e0 == cudaSuccess) e0 = dalloc(D, n64);
            if (e0 != cudaSuccess) { dfree(A); dfree(D); return cuda_fail(h, e0, "initial state"); }
            rc = accel_f64(h, h->d_init_U64, A, &launches);
            cudaError_t e1 = cudaSuccess;
            if (rc == SFM_OK) {
                if ((e1 = sfm::launch_start_delta(h->d_init_V64, A, dt, n64, D, st)) == cudaSuccess &&
                    (e1 = to_panel_any(mode, h->d_init_U64, r.U, h->nshots, h->nstate, st)) == cudaSuccess &&
                    (e1 = to_panel_any(mode, D, r.dU, h->nshots, h->nstate, st)) == cudaSuccess)
                    e1 = cudaStreamSynchronize(st);
                launches += 3;
            }
            dfree(A);
            dfree(D);
            if (rc != SFM_OK) return rc;
            if (e1 != cudaSuccess) return cuda_fail(h, e1, "initial state");
        }
    }
    if (flags & SFM_ENERGY) {
        x->energy.assign(2 * (size_t)h->nshots, 0.0);
        rc = energy_of_panel(h, mode, r.U, r.dU, h->nshots, dt, x->energy.data());
        if (rc != SFM_OK) return rc;
    }
    rc = ensure_ustep(h);
    if (rc != SFM_OK) return rc;
    int grid = 0, ncw = 0, nstage = 0;
    rc = panel_setup(h, mode, &grid, &ncw, &nstage);
    if (rc != SFM_OK) return rc;
    CK(h, cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), st));
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    CK(h, cudaMemsetAsync(x->d_bad, 0, sizeof(int), st));
    sfm::PanelParams p{};
    p.nsub = h->nsub; p.ngroups = ngroups; p.nsteps = nsteps;
    p.ncw = ncw; p.nstage = nstage; p.bmax = h->bmax; p.rpmax = c.rpmax;
    p.nstate = h->nstate; p.nmail = h->nmail;
    p.task_ptr = x->d_task_ptr; p.task = x->d_task;
    p.coef_off = mode == 2 ? c.d_coef2_off : c.d_coef_off;
    p.coef = mode == 2 ? c.coef2 : c.coef;
    p.state_off = h->d_state_off; p.mail_off = h->d_mail_off; p.frow = h->d_frow;
    p.H = mode == 2 ? c.H2 : c.H;
    p.src_off = c.d_src_off; p.src = c.src; p.wavelet = r.wav;
    p.sub_rp_ptr = c.d_sub_rp_ptr; p.sub_rp = c.d_sub_rp; p.rp_off = h->d_rp_off;
    p.rrows = mode == 2 ? c.rrows2 : c.rrows;
    p.nrpairs = h->nrpairs; p.partial = r.partial;
    p.U = r.U; p.dU = r.dU; p.mail0 = r.mail[0]; p.mail1 = r.mail[1];
    p.dt2 = (float)(dt * dt);
    p.dt2lo = (float)(dt * dt - (double)p.dt2);
    p.bar = h->d_bar; p.err = h->d_err; p.timeout_ns = x->timeout_ns; p.skip_arrive = x->skip_arrive;
    p.ustep = x->d_ustep;
    CK(h, cudaEventRecord(x->ev0, st));
    cudaError_t e = sfm::launch_panel(mode, p, grid, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "panel kernel launch");
    ++launches;
    CK(h, cudaEventRecord(x->ev1, st));
    if (h->nrpairs > 0) {
        if (mode == 2)
            CK(h, sfm::launch_panel_traces2(r.partial, h->d_rec_ptr, h->d_rec_pairs, h->nshots, nsteps,
                                            h->nrec, h->nrpairs, d_traces, x->d_bad, st));
        else
            CK(h, sfm::launch_panel_traces(r.partial, h->d_rec_ptr, h->d_rec_pairs, h->nshots, nsteps,
                                           h->nrec, h->nrpairs, d_traces, x->d_bad, st));
    } else {
        CK(h, cudaMemsetAsync(d_traces, 0, ntr * sizeof(double), st));
    }
    ++launches;
    int herr = 0, bad = 0;
    CK(h, cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaMemcpyAsync(&bad, x->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!(flags & SFM_DEVICE_PTR))
        CK(h, cudaMemcpyAsync(traces, d_traces, ntr * sizeof(double), cudaMemcpyDeviceToHost, st));
    int ustep = INT_MAX;
    CK(h, cudaMemcpyAsync(&ustep, x->d_ustep, sizeof(int), cudaMemcpyDeviceToHost, st));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "panel stepping");
    h->last_launches = launches;
    x->info.unstable_step = ustep == INT_MAX ? -1 : ustep;
    if (kernel_ms) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, x->ev0, x->ev1);
        *kernel_ms = ms;
    }
    if (herr == SFM_ERR_TIMEOUT) return fail(h, SFM_ERR_TIMEOUT, "device-wide barrier timed out");
    if (herr == SFM_ERR_UNSTABLE)
        return fail(h, SFM_ERR_UNSTABLE, "unstable: the state ran away at step " +
                                             std::to_string(x->info.unstable_step) +
                                             " (time step above the CFL limit?)");
    if (herr != 0) return fail(h, herr, "device error during stepping");
    if (bad) return fail(h, SFM_ERR_UNSTABLE, "non-finite traces (time step above the CFL limit?)");
    if ((flags & SFM_ENERGY) && !zero_source) {
        rc = energy_of_panel(h, mode, r.U, r.dU, h->nshots, dt, x->energy.data() + h->nshots);
        if (rc != SFM_OK) return rc;
    }
    return SFM_OK;
}

extern "C" int sfm_run(sfm_handle* h, int precision, double dt, int nsteps, const double* wavelet,
                       double* traces, int flags, double* kernel_ms) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (!h->have_coef || !h->have_src || !h->have_rec)
        return fail(h, SFM_ERR_STATE, "sfm_run: coefficients, sources and receivers must be set");
    if (nsteps < 1 || !(dt > 0.0) || !wavelet || !traces)
        return fail(h, SFM_ERR_ARG, "sfm_run: bad arguments");
    if ((flags & SFM_ENERGY) && h->bmax > sfm::BMAX_NARROW)
        return fail(h, SFM_ERR_ARG, "sfm_run: the energy report takes blocks up to 64 wide");
    CK(h, cudaSetDevice(h->device));
    sfm_ext* x = ext(h);
    x->ck_prec = -1;
    const auto t0 = std::chrono::steady_clock::now();
    x->info = sfm_run_info{precision, nsteps, h->nshots, 0, 0.0, 0.0, 0, -1, 0};
    if (!(flags & SFM_ENERGY)) x->energy.clear();
    double kms = 0.0;
    kernel_ms = kernel_ms ? kernel_ms : &kms;
    *kernel_ms = 0.0;
    int rc;
    if (precision == SFM_FP64)
        rc = run_impl<sfm::PolF64>(h, dt, nsteps, wavelet, traces, flags, kernel_ms);
    else if (precision == SFM_FP32)
        rc = run_impl<sfm::PolF32>(h, dt, nsteps, wavelet, traces, flags, kernel_ms);
    else if (precision == SFM_FP32X2)
        rc = run_impl<sfm::PolF32x2>(h, dt, nsteps, wavelet, traces, flags, kernel_ms);
    else if (precision == SFM_FP32F)
        rc = run_impl<sfm::PolF32F>(h, dt, nsteps, wavelet, traces, flags, kernel_ms);
    else if (precision == SFM_FP32FX2)
        rc = run_impl<sfm::PolF32Fx2>(h, dt, nsteps, wavelet, traces, flags, kernel_ms);
    else if (is_panel(precision))
        rc = run_panel_impl(h, panel_mode_of(precision), dt, nsteps, wavelet, traces, flags, kernel_ms);
    else if (precision == SFM_BF16)
        return fail(h, SFM_ERR_ARG, "sfm_run: BF16 products are not built (an 8-bit significand "
                                    "is coarser than TF32's 11 bits, with which the factored "
                                    "stepping of deep ROMs already diverges)");
    else
        return fail(h, SFM_ERR_ARG, "sfm_run: unknown precision");
    x->info.status = rc;
    x->info.launches = h->last_launches;
    x->info.kernel_ms = *kernel_ms;
    x->info.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    x->info.energy = (rc == SFM_OK && (flags & SFM_ENERGY)) ? 1 : 0;
    if (rc == SFM_OK) {
        x->ck_prec = precision;
        x->ck_steps = nsteps;
        x->ck_nshots = h->nshots;
    }
    return rc;
}

extern "C" int sfm_run_report(const sfm_handle* h, sfm_run_info* info, double* energy, int capacity) {
    if (!h || !info) return fail(nullptr, SFM_ERR_ARG, "sfm_run_report: bad arguments");
    const sfm_ext* x = reinterpret_cast<const sfm_ext*>(h->scratch);
    *info = x->info;
    if (energy && x->info.energy) {
        if (capacity < (int)x->energy.size())
            return fail(nullptr, SFM_ERR_ARG, "sfm_run_report: energy capacity below 2 * nshots");
        std::copy(x->energy.begin(), x->energy.end(), energy);
    }
    return SFM_OK;
}

// Shape search for the stepping kernel: every candidate (consumer warps,
// ring stages) that fits the shared memory runs a zero-source probe of
// `nsteps` steps twice (the first run warms caches and the piece table),
// timed by events around the step kernel alone; the fastest shape is kept
// for `precision` on this handle.  The state stays zero, so no candidate
// can go unstable, and the timing does not depend on the values.
template <class P>
static int autotune_impl(sfm_handle* h, int nsteps, int* ncw_out, int* nstage_out, double* us_out) {
    static const int kNcw[] = {2, 4, 6, 8};
    static const int kStage[] = {2, 3, 4, 6, 8, 12, 16};
    sfm_ext* x = ext(h);
    const int id = prec_id(P{});
    const int ncw0 = x->ncw[id], nst0 = x->nstage[id];
    std::vector<double> wav((size_t)h->nshots * nsteps, 0.0);
    std::vector<double> tr((size_t)h->nshots * h->nrec * (nsteps + 1));
    double best = 1e300;
    int bn = ncw0, bs = nst0;
    for (int nc : kNcw) {
        if (nc > sfm::step_max_ncw<P>()) continue;       // beyond the kernel's launch bounds
        for (int ns : kStage) {
            if (P::factored && ns % nc != 0) continue;   // see step_setup
            int gmax = 0;
            if (sfm::step_max_grid<P>(nc, sfm::step_smem_bytes<P>(h->kmax, h->bmax, ns), &gmax) != 0 ||
                gmax < 1)
                continue;
            x->ncw[id] = nc;
            x->nstage[id] = ns;
            double ms = 0.0, ms2 = 0.0;
            int rc = run_impl<P>(h, 1.0, nsteps, wav.data(), tr.data(), 0, &ms);
            if (rc == SFM_OK) rc = run_impl<P>(h, 1.0, nsteps, wav.data(), tr.data(), 0, &ms2);
            if (rc != SFM_OK) { x->ncw[id] = ncw0; x->nstage[id] = nst0; return rc; }
            ms = std::min(ms, ms2);
            if (ms < best) { best = ms; bn = nc; bs = ns; }
        }
    }
    x->ncw[id] = bn;
    x->nstage[id] = bs;
    if (ncw_out) *ncw_out = bn;
    if (nstage_out) *nstage_out = bs;
    if (us_out) *us_out = best * 1e3 / nsteps;
    return SFM_OK;
}

// The same search for the panel modes: 16-shot groups per task (consumer
// warps) in {1, 2, 4, 8} up to the number of groups, ring stages in
// {2, 3, 4, 6, 8}, each timed on zero-source probes from rest.
static int autotune_panel(sfm_handle* h, int mode, int nsteps, int* ncw_out, int* nstage_out,
                          double* us_out) {
    static const int kNcw[] = {1, 2, 4, 8};
    static const int kStage[] = {2, 3, 4, 6, 8};
    sfm_ext* x = ext(h);
    int rc = prepare_panel(h, mode);
    if (rc != SFM_OK) return rc;
    const int slot = panel_slot(mode);
    const int ncw0 = x->pncw[slot], nst0 = x->pnstage[slot];
    std::vector<double> tr((size_t)h->nshots * h->nrec * (nsteps + 1));
    double best = 1e300;
    int bn = ncw0, bs = nst0;
    for (int nc : kNcw) {
        if (nc > 1 && nc > x->pc.ngroups) continue;
        if (nc > sfm::panel_max_ncw(mode)) continue;
        for (int ns : kStage) {
            int gmax = 0;
            if (sfm::panel_max_grid(mode, nc, sfm::panel_smem_bytes(mode, nc, ns, h->bmax, x->pc.rpmax), &gmax) != 0 ||
                gmax < 1)
                continue;
            x->pncw[slot] = nc;
            x->pnstage[slot] = ns;
            double ms = 0.0, ms2 = 0.0;
            rc = run_panel_impl(h, mode, 1.0, nsteps, nullptr, tr.data(), 0, &ms, true);
            if (rc == SFM_OK) rc = run_panel_impl(h, mode, 1.0, nsteps, nullptr, tr.data(), 0, &ms2, true);
            if (rc != SFM_OK) { x->pncw[slot] = ncw0; x->pnstage[slot] = nst0; return rc; }
            ms = std::min(ms, ms2);
            if (ms < best) { best = ms; bn = nc; bs = ns; }
        }
    }
    x->pncw[slot] = bn;
    x->pnstage[slot] = bs;
    if (ncw_out) *ncw_out = bn;
    if (nstage_out) *nstage_out = bs;
    if (us_out) *us_out = best * 1e3 / nsteps;
    return SFM_OK;
}

extern "C" int sfm_autotune(sfm_handle* h, int precision, int nsteps, int* ncw, int* nstage,
                            double* us_per_step) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (!h->have_coef || !h->have_src || !h->have_rec)
        return fail(h, SFM_ERR_STATE, "sfm_autotune: coefficients, sources and receivers must be set");
    if (nsteps < 1) return fail(h, SFM_ERR_ARG, "sfm_autotune: nsteps < 1");
    CK(h, cudaSetDevice(h->device));
    ext(h)->ck_prec = -1;                  // the probes overwrite the run buffers
    // the probes step from rest (dt = 1 is far above the stability limit
    // for any nonzero state); an initial or restored state is kept for the
    // next sfm_run
    const bool had_init = h->have_init;
    h->have_init = false;
    int rc;
    if (precision == SFM_FP64) rc = autotune_impl<sfm::PolF64>(h, nsteps, ncw, nstage, us_per_step);
    else if (precision == SFM_FP32) rc = autotune_impl<sfm::PolF32>(h, nsteps, ncw, nstage, us_per_step);
    else if (precision == SFM_FP32X2)
        rc = autotune_impl<sfm::PolF32x2>(h, nsteps, ncw, nstage, us_per_step);
    else if (precision == SFM_FP32F)
        rc = autotune_impl<sfm::PolF32F>(h, nsteps, ncw, nstage, us_per_step);
    else if (precision == SFM_FP32FX2)
        rc = autotune_impl<sfm::PolF32Fx2>(h, nsteps, ncw, nstage, us_per_step);
    else if (is_panel(precision))
        rc = autotune_panel(h, panel_mode_of(precision), nsteps, ncw, nstage, us_per_step);
    else
        rc = fail(h, SFM_ERR_ARG, "sfm_autotune: unknown precision");
    h->have_init = had_init;
    return rc;
}

// ---------------------------------------------------------------------------
// Checkpoint and restore of the stepping state.  Blob layout (native byte
// order): 8 int64 header words {magic, version, nshots, nstate, nsub,
// topology fingerprint, time steps behind the state, precision}, then U^N
// and delta^N, nshots * nstate FP64 each, in the state layout.

namespace {

constexpr long long kCkMagic = 0x54504b434d4653LL;   // "SFMCKPT" little-endian
constexpr long long kCkVersion = 1;

long long topology_fingerprint(const sfm_handle* h) {
    unsigned long long f = 1469598103934665603ull;     // FNV-1a over k, b, m, nbr
    auto mix = [&](long long v) {
        for (int i = 0; i < 8; ++i) {
            f ^= (unsigned long long)((v >> (8 * i)) & 0xff);
            f *= 1099511628211ull;
        }
    };
    for (int s = 0; s < h->nsub; ++s) {
        mix(h->k[s]);
        mix(h->b[s]);
        for (int q = 0; q < 6; ++q) {
            mix(h->mface[s * 6 + q]);
            mix(h->nbr[s * 6 + q]);
        }
    }
    return (long long)(f >> 1);
}

double to_f64(double v) { return v; }
double to_f64(float v) { return (double)v; }
double to_f64(float2 v) { return (double)v.x + (double)v.y; }

template <typename T>
cudaError_t fetch_state(const T* d_U, const T* d_dU, size_t n, cudaStream_t st, double* U,
                        double* dU) {
    std::vector<T> a(n), b(n);
    cudaError_t e = cudaMemcpyAsync(a.data(), d_U, n * sizeof(T), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.data(), d_dU, n * sizeof(T), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (size_t i = 0; i < n; ++i) {
        U[i] = to_f64(a[i]);
        dU[i] = to_f64(b[i]);
    }
    return cudaSuccess;
}

}  // namespace

extern "C" int sfm_checkpoint(sfm_handle* h, void* buf, size_t* bytes) {
    if (!h || !bytes) return fail(h, SFM_ERR_ARG, "sfm_checkpoint: bad arguments");
    sfm_ext* x = ext(h);
    if (x->ck_prec < 0) return fail(h, SFM_ERR_STATE, "sfm_checkpoint: no stepping state");
    const size_t n = (size_t)x->ck_nshots * h->nstate;
    const size_t need = 8 * sizeof(long long) + 2 * n * sizeof(double);
    const size_t cap = *bytes;
    *bytes = need;
    if (!buf) return SFM_OK;
    if (cap < need) return fail(h, SFM_ERR_ARG, "sfm_checkpoint: buffer too small");
    CK(h, cudaSetDevice(h->device));
    long long* hd = static_cast<long long*>(buf);
    hd[0] = kCkMagic; hd[1] = kCkVersion; hd[2] = x->ck_nshots; hd[3] = h->nstate;
    hd[4] = h->nsub; hd[5] = topology_fingerprint(h); hd[6] = x->ck_steps; hd[7] = x->ck_prec;
    double* U = reinterpret_cast<double*>(hd + 8);
    double* dU = U + n;
    const int slot = x->ck_steps % 4;                   // U^n lives in buffer n mod 4
    cudaError_t e;
    if (is_panel(x->ck_prec)) {
        // panel state (updated in place) back to the state layout
        const int mode = panel_mode_of(x->ck_prec);
        double *dUx = nullptr, *dDx = nullptr;
        e = dalloc(dUx, n);
        if (e == cudaSuccess) e = dalloc(dDx, n);
        if (e == cudaSuccess) e = from_panel_any(mode, x->pb.U, dUx, x->ck_nshots, h->nstate, h->stream);
        if (e == cudaSuccess) e = from_panel_any(mode, x->pb.dU, dDx, x->ck_nshots, h->nstate, h->stream);
        if (e == cudaSuccess) e = fetch_state(dUx, dDx, n, h->stream, U, dU);
        dfree(dUx);
        dfree(dDx);
    } else if (x->ck_prec == SFM_FP64)
        e = fetch_state(x->r64.U[slot], x->r64.dU, n, h->stream, U, dU);
    else if (x->ck_prec == SFM_FP32X2 || x->ck_prec == SFM_FP32FX2)
        e = fetch_state(x->r2.U[slot], x->r2.dU, n, h->stream, U, dU);
    else
        e = fetch_state(x->r32.U[slot], x->r32.dU, n, h->stream, U, dU);
    if (e != cudaSuccess) return cuda_fail(h, e, "sfm_checkpoint");
    return SFM_OK;
}

extern "C" int sfm_restore(sfm_handle* h, const void* buf, size_t bytes) {
    if (!h || !buf || bytes < 8 * sizeof(long long))
        return fail(h, SFM_ERR_ARG, "sfm_restore: bad arguments");
    if (h->nsub == 0) return fail(h, SFM_ERR_STATE, "sfm_restore: no topology");
    const long long* hd = static_cast<const long long*>(buf);
    if (hd[0] != kCkMagic || hd[1] != kCkVersion)
        return fail(h, SFM_ERR_ARG, "sfm_restore: not a checkpoint of this format");
    const long long nshots = hd[2];
    if (nshots < 1 || hd[3] != h->nstate || hd[4] != h->nsub || hd[5] != topology_fingerprint(h))
        return fail(h, SFM_ERR_ARG, "sfm_restore: checkpoint of a different topology");
    const size_t n = (size_t)nshots * h->nstate;
    if (bytes != 8 * sizeof(long long) + 2 * n * sizeof(double))
        return fail(h, SFM_ERR_ARG, "sfm_restore: size does not match the header");
    CK(h, cudaSetDevice(h->device));
    const double* U = reinterpret_cast<const double*>(hd + 8);
    CK(h, upload(h->d_init_U64, U, n, h->stream));
    CK(h, upload(h->d_init_V64, U + n, n, h->stream));
    h->init_nshots = (int)nshots;
    h->have_init = true;
    h->init_delta = true;
    return SFM_OK;
}

// Largest eigenvalue of MM^{-1} KK.  One FP64 step of the stepping kernel
// from state X with zero increment, zero source and dt = 1 leaves the
// increment equal to -MM^{-1} KK X, and with Kx set the kernel also stores
// -KK X (the flux sums before the mass blocks).  MM^{-1} KK is self-adjoint
// in the MM inner product, so the iteration keeps q and r = MM q together
// (r_next = KK q is MM times q_next = MM^{-1} KK q) and reports the Rayleigh
// quotient q^T KK q / q^T MM q, which converges twice as fast as the plain
// ratio of norms and never exceeds lambda_max.  Shared face blocks are held
// once per side, so inner products weigh their entries by 1/2.
extern "C" int sfm_cfl_dt(sfm_handle* h, int iters, double* lambda_max, double* dt_cfl) {
    if (!h) return fail(nullptr, SFM_ERR_ARG, "NULL handle");
    if (!h->have_coef) return fail(h, SFM_ERR_STATE, "sfm_cfl_dt: no coefficients");
    if (iters < 1) return fail(h, SFM_ERR_ARG, "sfm_cfl_dt: iters < 1");
    CK(h, cudaSetDevice(h->device));
    sfm_ext* x = ext(h);
    // sources/receivers are not needed: convert what exists (possibly empty)
    int rc = prepare<sfm::PolF64>(h);
    if (rc != SFM_OK) return rc;
    Cache<double>& c = x->c64;
    cudaStream_t st = h->stream;
    const size_t n = (size_t)h->nstate;
    double *U[3] = {nullptr, nullptr, nullptr}, *dU = nullptr, *mail0 = nullptr, *mail1 = nullptr,
           *wav = nullptr, *X = nullptr, *ss = nullptr, *Kx = nullptr, *R = nullptr, *W = nullptr,
           *num = nullptr, *den = nullptr;
    long long* soff = nullptr;
    auto cleanup = [&]() {
        for (auto& u : U) dfree(u);
        dfree(dU); dfree(mail0); dfree(mail1); dfree(wav); dfree(X); dfree(ss); dfree(soff);
        dfree(Kx); dfree(R); dfree(W); dfree(num); dfree(den);
    };
#define CKC(call)                                                              \
    do {                                                                       \
        cudaError_t e__ = (call);                                              \
        if (e__ != cudaSuccess) { cleanup(); return cuda_fail(h, e__, #call); } \
    } while (0)
    for (auto& u : U) CKC(dalloc(u, n));
    CKC(dalloc(dU, n));
    CKC(dalloc(Kx, n));
    CKC(dalloc(R, n));
    CKC(dalloc(W, n));
    CKC(dalloc(mail0, (size_t)h->nmail));
    CKC(dalloc(mail1, (size_t)h->nmail));
    CKC(dalloc(wav, 1));
    CKC(dalloc(X, n));
    CKC(dalloc(ss, 1));
    CKC(dalloc(num, 1));
    CKC(dalloc(den, 1));
    std::vector<long long> none(h->nsub, -1);
    CKC(upload(soff, none.data(), none.size(), st));
    // start vector: pseudo-random (a symmetric start would stay in the
    // symmetric subspace of a symmetric problem), equal on both copies of a
    // shared face block (keyed by the lower-numbered side)
    auto mix = [](unsigned long long z) {
        z += 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    std::vector<double> x0(n), wts(n, 1.0);
    for (int s = 0; s < h->nsub; ++s) {
        const int b = h->b[s];
        for (int t = 0; t < h->k[s] * b; ++t) {
            unsigned long long key;
            if (t < b) {
                int f = 0;
                while (t >= h->face_off[s * 7 + f + 1]) ++f;
                const int nb = h->nbr[s * 6 + f], i = t - h->face_off[s * 7 + f];
                const int lo = (nb >= 0 && nb < s) ? nb : s;
                const int flo = (lo == s) ? f : (f ^ 1);
                key = ((unsigned long long)lo * 8 + flo) * 4096 + i;
                if (nb >= 0) wts[h->state_off[s] + t] = 0.5;
            } else {
                key = (1ull << 62) + (unsigned long long)h->state_off[s] + t;
            }
            x0[h->state_off[s] + t] = 0.5 + mix(key);
        }
    }
    CKC(cudaMemcpyAsync(X, x0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    CKC(cudaMemcpyAsync(W, wts.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    CKC(cudaMemsetAsync(wav, 0, sizeof(double), st));

    sfm::StepParams<double> p{};
    p.nsub = h->nsub; p.nshots = 1; p.nunits = h->nsub; p.nsteps = 1;
    p.kmax = h->kmax; p.bmax = h->bmax;
    p.sub_b = h->d_b; p.sub_k = h->d_k; p.coef_off = h->d_tcoef_off; p.coef = c.coef;
    p.face_off = h->d_face_off; p.nbr = h->d_nbr; p.H_off = h->d_H_off; p.H = c.H;
    p.state_off = h->d_state_off; p.state_stride = h->nstate;
    for (int i = 0; i < 3; ++i) p.U[i] = U[i];
    p.U[3] = nullptr;                                // one step: U[0] -> U[1]
    p.rctr = nullptr;                                // no receivers
    p.dU = dU;
    p.mail_off = h->d_mail_off; p.mail_stride = h->nmail; p.mail0 = mail0; p.mail1 = mail1;
    p.src_off = soff; p.src = c.src; p.wavelet = wav;
    p.nrec = 0; p.nrpairs = 0; p.rp_sub = nullptr; p.rp_off = nullptr; p.rrows = nullptr;
    p.partial = nullptr;
    p.dt2 = 1.0;
    p.bar = h->d_bar; p.err = h->d_err; p.timeout_ns = x->timeout_ns; p.skip_arrive = -1;
    p.Kx = Kx;
    int grid = 0;
    {
        const int r2 = step_setup<sfm::PolF64>(h, h->nsub, nullptr, p, &grid);
        if (r2 != SFM_OK) { cleanup(); return r2; }
    }
    auto apply = [&](const double* in) -> cudaError_t {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(U[0], in, n * sizeof(double), cudaMemcpyDeviceToDevice, st))) return e;
        if ((e = cudaMemsetAsync(dU, 0, n * sizeof(double), st))) return e;
        if ((e = cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), st))) return e;
        if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st))) return e;
        return sfm::launch_step<sfm::PolF64>(p, grid, st);
    };
    // q_1 = -MM^{-1} KK 1 (in dU), r_1 = MM q_1 = -KK 1 (in Kx)
    CKC(apply(X));
    CKC(sfm::launch_sumsq(dU, n, ss, st));
    CKC(sfm::launch_scale(dU, X, n, ss, st));
    CKC(sfm::launch_scale(Kx, R, n, ss, st));
    for (int it = 0; it < iters; ++it) {
        CKC(apply(X));                                   // dU = -A q, Kx = -KK q
        CKC(sfm::launch_wdot(X, Kx, W, n, num, st));     // -q^T KK q
        CKC(sfm::launch_wdot(X, R, W, n, den, st));      //  q^T MM q
        CKC(sfm::launch_sumsq(dU, n, ss, st));
        CKC(sfm::launch_scale(dU, X, n, ss, st));        // q <- -A q / |A q|
        CKC(sfm::launch_scale(Kx, R, n, ss, st));        // r <- MM q (same scale)
    }
    double hn = 0.0, hd = 1.0;
    int herr = 0;
    CKC(cudaMemcpyAsync(&hn, num, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(&hd, den, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
#undef CKC
    cleanup();
    if (herr != 0) return fail(h, herr, "sfm_cfl_dt: device error");
    const double lam = -hn / hd;
    if (!(lam > 0.0)) return fail(h, SFM_ERR_UNSTABLE, "sfm_cfl_dt: non-positive Rayleigh quotient");
    if (lambda_max) *lambda_max = lam;
    if (dt_cfl) *dt_cfl = 2.0 / std::sqrt(lam);
    return SFM_OK;
}
