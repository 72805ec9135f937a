// Internal declarations shared by the translation units of libsfm.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/sfm.h"
#include "numeric.cuh"

#define SFM_MAX_FACE_M 32      // largest m on one face (H_f kernel smem)

namespace sfm {

// Device-side description of the coupled ROM set in one compute precision
// (T = the policy's storage type).  All offsets are element offsets into
// the arrays they index.
template <typename T>
struct StepParams {
    int nsub, nshots, nunits, nsteps;
    int kmax, bmax;
    const int* sub_b;            // [nsub]
    const int* sub_k;            // [nsub]
    const long long* coef_off;   // [nsub] -> per level j: Gamma_j tiles, Gammahat_j tiles
    const T* coef;               // 8x8-tile packed upper triangles (see pack_tiles_kernel)
    const float* fcoef;          // factored policies: FP32 lower Cholesky factor tiles
                                 // (see factor_tiles_kernel), same offsets
    const int* face_off;         // [nsub*7] start of face f inside the b-vector
    const int* nbr;              // [nsub*6]
    const long long* H_off;      // [nsub*6] -> m_f*m_f block, or -1
    const T* H;
    const long long* state_off;  // [nsub] offset of the k*b state of shot 0
    long long state_stride;      // per shot
    T* U[4];                     // state buffers, U^n lives in U[n % 4]
    T* dU;                       // increments (one buffer, updated in place)
    const long long* mail_off;   // [nsub] offset of the b-vector of shot 0
    long long mail_stride;       // per shot
    T* mail0;
    T* mail1;
    const long long* src_off;    // [nshots*nsub] offset of (k*b) source rows, -1 if none
    const T* src;
    const T* wavelet;            // [nshots][nsteps]
    int nrec, nrpairs;
    const int* rp_sub;           // [nrpairs] subdomain of each receiver pair
    const long long* rp_off;     // [nrpairs] offset of its (k*b) row
    const T* rrows;
    T* partial;                  // [nshots][nsteps+1][nrpairs]
    unsigned* rctr;              // [nsteps+1] readout item counters, zero at launch
    double dt2;
    unsigned int* bar;           // grid barrier counter (zeroed before launch)
    int* err;                    // device error word (0 = ok)
    unsigned long long timeout_ns;
    int skip_arrive;             // test hook: this block skips its barrier arrival (-1: none)
    T* Kx;                       // optional: receives -KK U (the flux sums before the mass
                                 // blocks are applied), state layout; NULL when stepping
    int ncw, nstage;             // consumer warps per block, shared-memory ring stages
    const int* piece_ptr;        // [grid+1] pieces of each block
    const int4* prec;            // [2*npieces] piece records (see piece_records)
    const int4* frow;            // [mail layout] face rows (see face_rows)
    const int4* rtab;            // [nrpairs] receiver pairs (see readout_table)
    int stage_v4;                // factored path: stage piece state with 16-byte copies
                                 // (every b a multiple of 4, FP32 storage)
    int* ustep;                  // instability sentinel: first step whose face update
                                 // was non-finite or beyond 1e30 (atomicMin), or NULL
};

// Launch bounds per policy.  The factored FP32 kernel is held to at most
// four consumer warps so that four blocks fit on an SM (96 registers a
// thread); the other policies take up to eight.
template <class P>
constexpr int step_max_ncw() { return std::is_same<P, PolF32F>::value ? 4 : 8; }
template <class P>
constexpr int step_max_threads() { return (step_max_ncw<P>() + 1) * 32; }
template <class P>
constexpr int step_min_blocks() { return std::is_same<P, PolF32F>::value ? 4 : 0; }   // 0: no minimum

// Block widths b = sum of a subdomain's six face counts.  The FP64, FP32 and
// two-float stepping, the offline builder and the projections take b up to
// BMAX_WIDE (the paper's m = 25 per face gives b = 150); the factored modes,
// the multi-shot panels, the energy report, the usable-depth cut, the
// surrogate and the allocation-free entry point keep each block's 8x8 tiles
// in one warp's registers or a 64-wide shared-memory array and take b up to
// BMAX_NARROW.
constexpr int BMAX_NARROW = 64;
constexpr int BMAX_WIDE = 192;

constexpr int PANEL_NCW_MAX = 8;   // 16-shot groups (consumer warps) per panel block
// the two-float panel kernel (mode 2) takes at most four consumer warps
// (255 registers a thread, one block of five warps per SM)
inline int panel_max_ncw(int mode) { return mode == 2 ? 4 : PANEL_NCW_MAX; }

// Device-side description of a multi-shot panel run (panel.cu): shots in
// groups of 16, every array FP32.  Offsets are in numbers.
struct PanelParams {
    int nsub, ngroups, nsteps;
    int ncw, nstage;             // consumer warps (groups per task), ring stages
    int bmax, rpmax;             // widest block, most receiver pairs of one subdomain
    long long nstate, nmail;     // numbers per shot in the state and in the face data
    const int* task_ptr;         // [grid+1] tasks of each block
    const int4* task;            // {subdomain, first group, groups, b | k << 8}
    const long long* coef_off;   // [nsub] first padded factor tile of the subdomain
    const float* coef;
    const long long* state_off;  // [nsub] (numbers per shot)
    const long long* mail_off;   // [nsub]
    const int4* frow;            // face rows (face_rows)
    const float* H;
    const long long* src_off;    // [ngroups*nsub] source panels of a unit, -1 if none
    const float* src;
    const float* wavelet;        // [ngroups*16][nsteps]
    const int* sub_rp_ptr;       // [nsub+1] receiver pairs of each subdomain ...
    const int* sub_rp;           // ... as pair indices
    const long long* rp_off;     // [nrpairs] start of the pair's k*b row
    const float* rrows;
    int nrpairs;
    float* partial;              // [ngroups][nsteps+1][nrpairs][16]
    float* U;                    // [ngroups][nstate][16]
    float* dU;
    float* mail0;
    float* mail1;
    float dt2;
    float dt2lo;                 // two-float mode: dt^2 - dt2 (rounded)
    unsigned int* bar;
    int* err;
    unsigned long long timeout_ns;
    int skip_arrive;
    int* ustep;                  // instability sentinel (as StepParams::ustep)
};

// panel launchers (panel.cu); mode 1 = 1xTF32, 3 = 3xTF32 products (FP32
// panels), 2 = two-float panels with compensated CUDA-core products
size_t panel_smem_bytes(int mode, int ncw, int nstage, int bmax, int rpmax);
int panel_max_grid(int mode, int ncw, size_t smem, int* grid_out);
cudaError_t launch_panel(int mode, const PanelParams& p, int grid, cudaStream_t st);
// LPT assignment of the tasks (subdomain, group chunk of at most ncw groups)
// to `grid` blocks by estimated cost
void build_panel_tasks(int nsub, int ngroups, const int* k_sub, const int* b_sub, int ncw,
                       int grid, std::vector<int>& ptr, std::vector<int4>& tasks);
// 64-float factor tiles -> 72-float padded tiles
cudaError_t launch_pad_tiles(const float* in, float* out, long long ntiles, cudaStream_t st);
// FP64 [nshots][n] -> FP32 panels [ngroups][n][16] (padded shots zero)
cudaError_t launch_to_panel(const double* in, float* out, int nshots, long long n, cudaStream_t st);
// FP32 panels -> FP64 [nshots][n]
cudaError_t launch_from_panel(const float* in, double* out, int nshots, long long n, cudaStream_t st);
// traces from the two-float partial sums of mode 2
cudaError_t launch_panel_traces2(const float* partial, const int* rec_ptr, const int* rec_pairs,
                                 int nshots, int nsteps, int nrec, int nrpairs, double* traces,
                                 int* bad, cudaStream_t st);
// two-float mode: FP64 [nshots][n] <-> [ngroups][n][16][hi, lo] (natural shot order)
cudaError_t launch_to_panel2(const double* in, float* out, int nshots, long long n, cudaStream_t st);
cudaError_t launch_from_panel2(const float* in, double* out, int nshots, long long n, cudaStream_t st);
// two-float padded tiles of every symmetric block (144 floats a tile)
cudaError_t launch_pack_sym2(const double* master, const long long* master_off, const long long* tile_off,
                             const int* sub_b, const int* sub_k, int nsub, float* out, cudaStream_t st);
// source rows of (shot, subdomain) pairs into their unit's panels:
// rows[off64[i] .. + len[i]) go to column dst[i] % 16 of out + dst[i] - dst[i] % 16
cudaError_t launch_src_panels(const double* rows, const long long* off64, const long long* dst,
                              const int* len, int npairs, float* out, cudaStream_t st);
// traces[q][r][n] = sum over the pairs of r of partial[q/16][n][pair][pos(q%16)]
cudaError_t launch_panel_traces(const float* partial, const int* rec_ptr, const int* rec_pairs,
                                int nshots, int nsteps, int nrec, int nrpairs, double* traces,
                                int* bad, cudaStream_t st);

// energy terms (energy.cu): out[(unit * kmax + j) * 2 + {0, 1}] =
// {delta_j^T Gammahat_j^{-1} delta_j, Delta_j(U)^T Gamma_j Delta_j(U - delta)}
// for U = U^{n+1}, delta = U^{n+1} - U^n in the state layout (FP64)
cudaError_t launch_energy_terms(const double* coef, const long long* coef_off, const int* sub_b,
                                const int* sub_k, int nsub, int kmax, int nshots, const double* U,
                                const double* D, long long stride, const long long* state_off,
                                double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_state_to_f64(const T* in, double* out, size_t n, cudaStream_t st);

// surrogate helpers (surrogate.cu): the network's block side and the (b, k)
// of its decoder (SFM_ERR_STATE without a decoder); the relative error of
// the transfer functions at sigma of `count` coefficient sets, and of their
// derivatives there, against real b x b references (Dref may be NULL)
int net_shape(const sfm_net* net, int* n, int* b, int* k);
int net_code_dim(const sfm_net* net);
cudaError_t sigma_check(const double* sets, int count, int b, int k, double sigma, const double* Sref,
                        const double* Dref, double* err, cudaStream_t st);

// launchers (step.cu); P is a number policy of numeric.cuh
template <class P>
cudaError_t launch_step(const StepParams<typename P::S>& p, int grid, cudaStream_t st);
template <class P>
int step_max_grid(int ncw, size_t smem, int* grid_out);
template <class P>
size_t step_smem_bytes(int kmax, int bmax, int nstage);
void build_pieces(int nunits, int nsub, const int* k_sub, int grid, std::vector<int>& ptr,
                  std::vector<int4>& pieces);
bool piece_records(const std::vector<int4>& pieces, int nsub, const int* k, const int* b,
                   const long long* state_off, const long long* src_off, const long long* mail_off,
                   std::vector<int4>& rec);
bool face_rows(int nsub, const int* b, const int* face_off, const int* nbr,
               const long long* H_off, const long long* mail_off, std::vector<int4>& rows);
bool readout_table(int nrpairs, const int* rp_sub, const long long* rp_off, const int* k,
                   const int* b, const long long* state_off, std::vector<int4>& tab);

cudaError_t launch_face_H(const double* coef, const long long* gh1_off, const int* sub_b,
                          const int* face_off, const int* nbr, const long long* H_off,
                          double* H, int nsub, int* err, cudaStream_t st);

template <class P>
cudaError_t launch_convert(const double* in, typename P::S* out, size_t n, cudaStream_t st);

// FP64 masters (per subdomain: Gamma_1..k then Gammahat_1..k, b x b row-major)
// -> 8x8-tile packed blocks in the policy's storage type.
template <class P>
cudaError_t launch_pack_tiles(const double* master, const long long* master_off,
                              const long long* tile_off, const int* sub_b, const int* sub_k,
                              int nsub, typename P::S* out, cudaStream_t st);

// FP64 masters -> FP32 lower Cholesky factors in 8x8 tiles (same offsets as
// launch_pack_tiles); *bad is set if a block the stepping uses is not
// positive definite.
cudaError_t launch_factor_tiles(const double* master, const long long* master_off,
                                const long long* tile_off, const int* sub_b, const int* sub_k,
                                int nsub, int kmax, float* out, int* bad, cudaStream_t st);

// number of 8x8 tiles kept of a b x b symmetric block (upper triangle of tiles)
__host__ __device__ inline long long sym_tiles(int b) {
    const long long nt = (b + 7) / 8;
    return nt * (nt + 1) / 2;
}

// power-iteration helpers (FP64)
cudaError_t launch_sumsq(const double* x, size_t n, double* out, cudaStream_t st);
cudaError_t launch_wdot(const double* x, const double* y, const double* w, size_t n, double* out,
                        cudaStream_t st);
cudaError_t launch_scale(const double* x, double* y, size_t n, const double* sumsq,
                         cudaStream_t st);
// out = dt * v - 0.5 * dt^2 * a (v NULL: zero velocity)
cudaError_t launch_start_delta(const double* v, const double* a, double dt, size_t n, double* out,
                               cudaStream_t st);

template <class P>
cudaError_t launch_reduce_traces(const typename P::S* partial, const int* rec_ptr,
                                 const int* rec_pairs, int nshots, int nsteps, int nrec,
                                 int nrpairs, double* traces, int* bad, cudaStream_t st);

void free_build(sfm_handle* h);
void set_global_error(const std::string& msg);   // text of sfm_last_error(NULL)
int set_topology_internal(sfm_handle* h, int nsub, const int* k_sub, const int* m_face,
                          const int* nbr);
int set_coeffs_device(sfm_handle* h, const double* d_coeffs);

}  // namespace sfm

// The opaque handle.
struct sfm_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = true;
    std::string err;
    int last_launches = 0;

    // topology (host copies)
    int nsub = 0;
    std::vector<int> k, b, mface, nbr, face_off;     // face_off: nsub*7
    std::vector<long long> coef_off, H_off, state_off, mail_off, tcoef_off;
    long long ncoef = 0, nH = 0, nstate = 0, nmail = 0, ntcoef = 0;
    int kmax = 0, bmax = 0;

    // device copies of the topology
    int *d_b = nullptr, *d_k = nullptr, *d_face_off = nullptr, *d_nbr = nullptr;
    long long *d_coef_off = nullptr, *d_H_off = nullptr, *d_state_off = nullptr,
              *d_mail_off = nullptr, *d_tcoef_off = nullptr;

    // FP64 master data
    double* d_coef64 = nullptr;
    double* d_H64 = nullptr;
    bool have_coef = false;

    int nshots = 0;
    std::vector<long long> src_off;                  // nshots*nsub
    long long nsrc = 0;
    double* d_src64 = nullptr;
    long long* d_src_off = nullptr;

    int nrec = 0, nrpairs = 0;
    std::vector<int> rp_sub, rp_rec;
    std::vector<long long> rp_off;
    long long nrrow = 0;
    double* d_rrows64 = nullptr;
    int *d_rp_sub = nullptr, *d_rec_ptr = nullptr, *d_rec_pairs = nullptr;
    long long* d_rp_off = nullptr;
    int4* d_frow = nullptr;            // face rows (face_rows), set with the topology
    // initial state (sfm_set_initial): U^0 and dU/dt(0) in the state layout,
    // FP64, for init_nshots shots (V NULL: zero velocity)
    double* d_init_U64 = nullptr;
    double* d_init_V64 = nullptr;
    int init_nshots = 0;
    bool have_init = false;
    bool init_delta = false;           // d_init_V64 holds delta^0 itself (sfm_restore)
    int4* d_rtab = nullptr;            // receiver pair table (readout_table)
    bool have_src = false, have_rec = false;

    // offline builder state (builder.cu), NULL until sfm_set_model
    void* build = nullptr;

    // scratch owned by the handle, grown on demand
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned int* d_bar = nullptr;
    int* d_err = nullptr;
};
