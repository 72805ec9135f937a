// sfm_run_static: the FP64 coupled stepping of sfm_run with no device
// allocation at all.  Its scratch memory (the layout tables, the tile-packed
// coefficient copy, the face coupling blocks, the state ring, the face data
// and the partial receiver sums) lives in one file-scope __device__ array of
// fixed size that every GPU loading the library holds until the process
// exits; inputs and outputs are device buffers the caller owns.
#include "sfm_internal.h"

#include <algorithm>
#include <string>
#include <vector>

#define SFM_STATIC_SCRATCH_BYTES (64ull << 20)   // 64 MiB

namespace {

__device__ __align__(256) unsigned char g_static_scratch[SFM_STATIC_SCRATCH_BYTES];

// failures are reported through sfm_last_error(NULL)
int sfail(int code, const std::string& msg) {
    sfm::set_global_error(msg);
    return code;
}

// Device address of the scratch array in the current context, looked up on
// every call (a table lookup once the module is loaded).  A cached address
// would go stale if the caller reset the device and the module were loaded
// again elsewhere.  With lazy module loading the first lookup on a device is
// the one that loads the module and so reserves the array.
int scratch_address(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
        return sfail(SFM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = static_cast<unsigned char*>(p);
    return SFM_OK;
}

// Makes `device` current for the scope and gives the caller's current device
// back on every return path.
struct DeviceScope {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int device) {
        err = cudaGetDevice(&prev);
        if (err != cudaSuccess) { prev = -1; return; }
        if (prev != device) err = cudaSetDevice(device);
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        const size_t at = off;
        off += (count ? count : 1) * sizeof(T);
        return at;
    }
};

}  // namespace

extern "C" int sfm_run_static(int device, void* stream, int nsub, const int* k_sub,
                              const int* m_face, const int* nbr, const double* coeffs, int nshots,
                              int nsrc_pairs, const int* src_shot, const int* src_sub,
                              const double* src_rows, int nrec, int nrec_pairs, const int* rec_id,
                              const int* rec_sub, const double* rec_rows, double dt, int nsteps,
                              const double* wavelet, double* traces) {
    using P = sfm::PolF64;
    if (nsub <= 0 || !k_sub || !m_face || !nbr || !coeffs || nshots < 1 || nsrc_pairs < 0 ||
        nrec < 1 || nrec_pairs < 0 || !(dt > 0.0) || nsteps < 1 || !wavelet || !traces ||
        (nsrc_pairs > 0 && (!src_shot || !src_sub || !src_rows)) ||
        (nrec_pairs > 0 && (!rec_id || !rec_sub || !rec_rows)))
        return sfail(SFM_ERR_ARG, "sfm_run_static: bad arguments");
    // ---- layout on the host (host memory only) ----
    std::vector<int> b(nsub), face_off(7 * (size_t)nsub), kk(k_sub, k_sub + nsub),
        nb(nbr, nbr + 6 * (size_t)nsub);
    std::vector<long long> coef_off(nsub), tcoef_off(nsub), gh1_off(nsub), H_off(6 * (size_t)nsub, -1),
        state_off(nsub), mail_off(nsub);
    long long co = 0, to = 0, ho = 0, so = 0, mo = 0;
    int kmax = 0, bmax = 0;
    for (int s = 0; s < nsub; ++s) {
        if (k_sub[s] < 1) return sfail(SFM_ERR_ARG, "sfm_run_static: k < 1");
        int bs = 0;
        for (int f = 0; f < 6; ++f) {
            const int m = m_face[s * 6 + f], t = nbr[s * 6 + f];
            if (m < 0 || m > SFM_MAX_FACE_M || t >= nsub || t < -1 || t == s ||
                (t >= 0 && (nbr[t * 6 + (f ^ 1)] != s || m_face[t * 6 + (f ^ 1)] != m)))
                return sfail(SFM_ERR_ARG, "sfm_run_static: inconsistent topology");
            face_off[s * 7 + f] = bs;
            if (m > 0) { H_off[s * 6 + f] = ho; ho += (long long)m * m; }
            bs += m;
        }
        face_off[s * 7 + 6] = bs;
        if (bs == 0 || bs > 64) return sfail(SFM_ERR_ARG, "sfm_run_static: block width outside 1..64");
        b[s] = bs;
        coef_off[s] = co;
        gh1_off[s] = co + (long long)k_sub[s] * bs * bs;
        co += 2LL * k_sub[s] * bs * bs;
        tcoef_off[s] = to;
        to += 2LL * k_sub[s] * sfm::sym_tiles(bs) * 64;
        state_off[s] = so;
        so += (long long)k_sub[s] * bs;
        mail_off[s] = mo;
        mo += bs;
        kmax = std::max(kmax, k_sub[s]);
        bmax = std::max(bmax, bs);
    }
    std::vector<long long> src_off((size_t)nshots * nsub, -1);
    long long sro = 0;
    for (int i = 0; i < nsrc_pairs; ++i) {
        const int q = src_shot[i], s = src_sub[i];
        if (q < 0 || q >= nshots || s < 0 || s >= nsub || src_off[(size_t)q * nsub + s] >= 0)
            return sfail(SFM_ERR_ARG, "sfm_run_static: bad source pair");
        src_off[(size_t)q * nsub + s] = sro;
        sro += (long long)k_sub[s] * b[s];
    }
    std::vector<int> rp_sub(nrec_pairs), cnt(nrec + 1, 0), pairs(nrec_pairs);
    std::vector<long long> rp_off(nrec_pairs);
    long long rro = 0;
    for (int i = 0; i < nrec_pairs; ++i) {
        const int r = rec_id[i], s = rec_sub[i];
        if (r < 0 || r >= nrec || s < 0 || s >= nsub) return sfail(SFM_ERR_ARG, "sfm_run_static: bad receiver pair");
        rp_sub[i] = s;
        rp_off[i] = rro;
        rro += (long long)k_sub[s] * b[s];
        cnt[r + 1]++;
    }
    for (int r = 0; r < nrec; ++r) cnt[r + 1] += cnt[r];
    {
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int i = 0; i < nrec_pairs; ++i) pairs[fill[rec_id[i]]++] = i;
    }
    // ---- block shape, grid and per-block pieces, sized on `device` ----
    if (device < 0) return sfail(SFM_ERR_ARG, "sfm_run_static: bad device");
    DeviceScope dev(device);
    if (dev.err != cudaSuccess)
        return sfail(SFM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(dev.err));
    const int ncw = 8, nstage = 6;
    int gmax = 0;
    if (sfm::step_max_grid<P>(ncw, sfm::step_smem_bytes<P>(kmax, bmax, nstage), &gmax) != 0)
        return sfail(SFM_ERR_ARG, "sfm_run_static: subdomain blocks too large for shared memory");
    long long levels = 0;
    for (int u = 0; u < nshots * nsub; ++u) levels += k_sub[u % nsub];
    const int grid = (int)std::max(1LL, std::min<long long>(gmax, levels));
    std::vector<int> piece_ptr;
    std::vector<int4> pieces, prec, frow, rtab;
    sfm::build_pieces(nshots * nsub, nsub, k_sub, grid, piece_ptr, pieces);
    if (!sfm::piece_records(pieces, nsub, k_sub, b.data(), state_off.data(), src_off.data(),
                            mail_off.data(), prec) ||
        !sfm::face_rows(nsub, b.data(), face_off.data(), nb.data(), H_off.data(), mail_off.data(), frow) ||
        !sfm::readout_table(nrec_pairs, rp_sub.data(), rp_off.data(), k_sub, b.data(),
                            state_off.data(), rtab))
        return sfail(SFM_ERR_ARG, "sfm_run_static: offsets beyond 32 bits");
    // ---- carve the scratch array ----
    Carve cv;
    const size_t o_pp = cv.take<int>(piece_ptr.size()), o_pc = cv.take<int4>(prec.size()),
                 o_fr = cv.take<int4>(frow.size()), o_rt = cv.take<int4>(rtab.size());
    const size_t o_b = cv.take<int>(nsub), o_k = cv.take<int>(nsub), o_fo = cv.take<int>(7 * (size_t)nsub),
                 o_nb = cv.take<int>(6 * (size_t)nsub), o_ho = cv.take<long long>(6 * (size_t)nsub),
                 o_to = cv.take<long long>(nsub), o_co = cv.take<long long>(nsub),
                 o_g1 = cv.take<long long>(nsub), o_so = cv.take<long long>(nsub),
                 o_mo = cv.take<long long>(nsub), o_sr = cv.take<long long>(src_off.size()),
                 o_rs = cv.take<int>(nrec_pairs), o_ro = cv.take<long long>(nrec_pairs),
                 o_rp = cv.take<int>(nrec + 1), o_pr = cv.take<int>(nrec_pairs);
    const size_t o_tiles = cv.take<double>((size_t)to), o_H = cv.take<double>((size_t)ho);
    size_t o_U[4];
    for (auto& u : o_U) u = cv.take<double>((size_t)nshots * so);
    const size_t o_dU = cv.take<double>((size_t)nshots * so), o_m0 = cv.take<double>((size_t)nshots * mo),
                 o_m1 = cv.take<double>((size_t)nshots * mo),
                 o_part = cv.take<double>((size_t)nshots * (nsteps + 1) * std::max(nrec_pairs, 1)),
                 o_bar = cv.take<unsigned int>(1), o_err = cv.take<int>(1), o_bad = cv.take<int>(1),
                 o_ctr = cv.take<unsigned int>((size_t)nsteps + 1);
    if (cv.off > SFM_STATIC_SCRATCH_BYTES)
        return sfail(SFM_ERR_ARG, "sfm_run_static: problem needs " + std::to_string(cv.off) +
                                      " bytes of scratch, the static limit is " +
                                      std::to_string(SFM_STATIC_SCRATCH_BYTES) + " bytes");
    // ---- device work: no allocation from here on ----
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != SFM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
#define SCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e__ = (call);                                                              \
        if (e__ != cudaSuccess) return sfail(SFM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)
    auto put = [&](size_t off, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    SCK(put(o_b, b.data(), b.size() * sizeof(int)));
    SCK(put(o_k, kk.data(), kk.size() * sizeof(int)));
    SCK(put(o_fo, face_off.data(), face_off.size() * sizeof(int)));
    SCK(put(o_nb, nb.data(), nb.size() * sizeof(int)));
    SCK(put(o_ho, H_off.data(), H_off.size() * sizeof(long long)));
    SCK(put(o_to, tcoef_off.data(), tcoef_off.size() * sizeof(long long)));
    SCK(put(o_co, coef_off.data(), coef_off.size() * sizeof(long long)));
    SCK(put(o_g1, gh1_off.data(), gh1_off.size() * sizeof(long long)));
    SCK(put(o_so, state_off.data(), state_off.size() * sizeof(long long)));
    SCK(put(o_mo, mail_off.data(), mail_off.size() * sizeof(long long)));
    SCK(put(o_sr, src_off.data(), src_off.size() * sizeof(long long)));
    SCK(put(o_rs, rp_sub.data(), rp_sub.size() * sizeof(int)));
    SCK(put(o_ro, rp_off.data(), rp_off.size() * sizeof(long long)));
    SCK(put(o_rp, cnt.data(), cnt.size() * sizeof(int)));
    SCK(put(o_pr, pairs.data(), pairs.size() * sizeof(int)));
    SCK(put(o_pp, piece_ptr.data(), piece_ptr.size() * sizeof(int)));
    SCK(put(o_pc, prec.data(), prec.size() * sizeof(int4)));
    SCK(put(o_fr, frow.data(), frow.size() * sizeof(int4)));
    SCK(put(o_rt, rtab.data(), rtab.size() * sizeof(int4)));
    auto at = [&](size_t off) { return (void*)(base + off); };
    // every call shares the array: clear what has to start at zero
    for (auto u : o_U) SCK(cudaMemsetAsync(at(u), 0, (size_t)nshots * so * sizeof(double), st));
    SCK(cudaMemsetAsync(at(o_dU), 0, (size_t)nshots * so * sizeof(double), st));
    SCK(cudaMemsetAsync(at(o_part), 0, (size_t)nshots * (nsteps + 1) * std::max(nrec_pairs, 1) * sizeof(double), st));
    SCK(cudaMemsetAsync(at(o_bar), 0, sizeof(unsigned int), st));
    SCK(cudaMemsetAsync(at(o_ctr), 0, ((size_t)nsteps + 1) * sizeof(unsigned int), st));
    SCK(cudaMemsetAsync(at(o_err), 0, sizeof(int), st));
    SCK(cudaMemsetAsync(at(o_bad), 0, sizeof(int), st));
    // face coupling blocks and the tile-packed coefficient copy
    SCK(sfm::launch_face_H(coeffs, (const long long*)at(o_g1), (const int*)at(o_b), (const int*)at(o_fo),
                           (const int*)at(o_nb), (const long long*)at(o_ho), (double*)at(o_H), nsub,
                           (int*)at(o_err), st));
    {
        // a face block that failed its Cholesky leaves its H_f unset: stop
        // before any stepping work is enqueued
        int herr0 = 0;
        SCK(cudaMemcpyAsync(&herr0, at(o_err), sizeof(int), cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        if (herr0 == SFM_ERR_NOT_SPD)
            return sfail(SFM_ERR_NOT_SPD, "sfm_run_static: a face block of Gammahat_1 is not SPD");
        if (herr0 != 0) return sfail(herr0, "sfm_run_static: device error in the face coupling");
    }
    SCK(sfm::launch_pack_tiles<P>(coeffs, (const long long*)at(o_co), (const long long*)at(o_to),
                                  (const int*)at(o_b), (const int*)at(o_k), nsub, (double*)at(o_tiles), st));
    sfm::StepParams<double> p{};
    p.nsub = nsub; p.nshots = nshots; p.nunits = nshots * nsub; p.nsteps = nsteps;
    p.kmax = kmax; p.bmax = bmax;
    p.sub_b = (const int*)at(o_b); p.sub_k = (const int*)at(o_k);
    p.coef_off = (const long long*)at(o_to); p.coef = (const double*)at(o_tiles);
    p.face_off = (const int*)at(o_fo); p.nbr = (const int*)at(o_nb);
    p.H_off = (const long long*)at(o_ho); p.H = (const double*)at(o_H);
    p.state_off = (const long long*)at(o_so); p.state_stride = so;
    for (int i = 0; i < 4; ++i) p.U[i] = (double*)at(o_U[i]);
    p.rctr = (unsigned*)at(o_ctr);
    p.dU = (double*)at(o_dU);
    p.mail_off = (const long long*)at(o_mo); p.mail_stride = mo;
    p.mail0 = (double*)at(o_m0); p.mail1 = (double*)at(o_m1);
    p.src_off = (const long long*)at(o_sr); p.src = src_rows; p.wavelet = wavelet;
    p.nrec = nrec; p.nrpairs = nrec_pairs; p.rp_sub = (const int*)at(o_rs);
    p.rp_off = (const long long*)at(o_ro); p.rrows = rec_rows; p.partial = (double*)at(o_part);
    p.dt2 = dt * dt;
    p.bar = (unsigned int*)at(o_bar); p.err = (int*)at(o_err);
    p.timeout_ns = 2000000000ull; p.skip_arrive = -1; p.Kx = nullptr;
    p.ncw = ncw; p.nstage = nstage;
    p.piece_ptr = (const int*)at(o_pp); p.prec = (const int4*)at(o_pc);
    p.frow = (const int4*)at(o_fr); p.rtab = (const int4*)at(o_rt);
    SCK(sfm::launch_step<P>(p, grid, st));
    SCK(sfm::launch_reduce_traces<P>((const double*)at(o_part), (const int*)at(o_rp), (const int*)at(o_pr),
                                     nshots, nsteps, nrec, nrec_pairs, traces, (int*)at(o_bad), st));
    int herr = 0, bad = 0;
    SCK(cudaMemcpyAsync(&herr, at(o_err), sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(&bad, at(o_bad), sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
#undef SCK
    if (herr == SFM_ERR_TIMEOUT) return sfail(SFM_ERR_TIMEOUT, "sfm_run_static: device-wide barrier timed out");
    if (herr == SFM_ERR_NOT_SPD) return sfail(SFM_ERR_NOT_SPD, "sfm_run_static: a face block of Gammahat_1 is not SPD");
    if (herr != 0) return sfail(herr, "sfm_run_static: device error");
    if (bad) return sfail(SFM_ERR_UNSTABLE, "sfm_run_static: non-finite traces");
    return SFM_OK;
}
