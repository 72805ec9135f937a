// Multi-shot coupled stepping with tensor-core block products (Algorithm 1
// stage 2; Eqs. 12, 18, 19), for runs with many shots: the shots of one
// subdomain are stepped together as panels of 16, so every S-fraction block
// streamed from memory is applied to 16 state vectors at once, a
// (16 x b) . (b x b) product on the tensor cores (mma.sync, TF32 inputs,
// FP32 accumulation) instead of 16 matrix-vector products.
//
// Each block is applied through its FP32 Cholesky factor, Gamma = L L^T, as
// in the factored FP32 mode (the product L (L^T x) stays positive
// semi-definite under any rounding of L).  With 3xTF32 products every factor
// and every input is split into a TF32 head and a TF32 tail (x = hi + lo)
// and hi.hi + hi.lo + lo.hi is accumulated in FP32, which keeps the products
// at FP32 accuracy; with 1xTF32 only hi.hi is kept (11 significant bits).
//
// Layout (all FP32):
//   state panel of (group g, subdomain s, level j): b x 16 numbers, row i of
//   shot c at (j*b + i)*16 + pos(c), pos(c) = 2*(c & 7) + (c >> 3), so that
//   shots c and c+8 of a row are adjacent; the panels of group g start at
//   g * nstate * 16, subdomain s at state_off[s] * 16 inside the group;
//   face data (mail) in the same form over the level-1 rows;
//   factor tiles: the lower-triangular 8x8 tiles of L, tile (I, J) (J <= I)
//   at I(I+1)/2 + J, 72 numbers per tile: row r at r*8 + 8*(r >> 2) (rows
//   4..7 shifted by 8 so that both fragment patterns below are free of
//   shared-memory bank conflicts); per level Gamma_j then Gammahat_j.
//
// Fragments of mma.m16n8k8 (g = lane / 4, t = lane % 4):
//   accumulator C (16 shots x 8 rows of one 8-row tile nt):
//     c0 = (shot g, row 8nt+2t), c1 = (shot g, row 8nt+2t+1),
//     c2 = (shot g+8, row 8nt+2t), c3 = (shot g+8, row 8nt+2t+1);
//   the same registers, read in the order {c0, c2, c1, c3}, are the A
//   fragment of k-tile nt when the reduction index of that tile is taken in
//   the order (2t, 2t+1) -> (t, t+4); the B fragment then holds the factor
//   entries of reduction rows 8kt+2t and 8kt+2t+1.  So the output of one
//   product is the input of the next with no data movement.
//
// Per time step n and (group, subdomain) unit, level by level (0-based j):
//   Delta_j = U_{j+1} - U_j,  phi_j = L_j (L_j^T Delta_j)            (Eq. 12)
//   j = 0:  mail = phi_0 + p_0 f(t_n)                          (step 2.1)
//   j >= 1: psi_j = phi_j - phi_{j-1} + p_j f(t_n),
//           a_j = Lh_j (Lh_j^T psi_j),  delta_j += dt^2 a_j,  U_j += delta_j
//                                                         (Eq. 19, step 2.2)
//   the receiver rows read U_j^n as it passes (readout of sample n);
// device-wide barrier; then per unit the face rows (step 2.3, Eq. 18):
//   a_f = H_f (mail_f(self) + mail_f(neighbour)), delta_0 += dt^2 a_f,
//   U_0 += delta_0.
// U and delta are updated in place: a unit's levels are read before they
// are written within the step, the face rows of a unit are written only by
// its own block, and the face data are double-buffered by step parity.
#include "sfm_internal.h"
#include "step_kernel.cuh"

#include <algorithm>
#include <climits>
#include <numeric>

namespace sfm {

constexpr int PTILE = 72;            // floats per padded 8x8 factor tile
constexpr int PANEL_BLOCK_MAX = (PANEL_NCW_MAX + 1) * 32;

__host__ __device__ inline long long tri_tiles(int b) {
    const long long nt = (b + 7) / 8;
    return nt * (nt + 1) / 2;
}

__device__ __forceinline__ unsigned f2tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// A fragments of a panel held in accumulator layout: head and tail words in
// the order {c0, c2, c1, c3} (see the file comment).
template <int NT, int MODE>
struct Frag {
    unsigned hi[NT][4];
    unsigned lo[MODE == 3 ? NT : 1][4];
};

template <int NT, int MODE>
__device__ __forceinline__ void split(const float (&v)[NT][4], Frag<NT, MODE>& f) {
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const float x[4] = {v[i][0], v[i][2], v[i][1], v[i][3]};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            f.hi[i][e] = f2tf32(x[e]);
            if constexpr (MODE == 3) f.lo[i][e] = f2tf32(x[e] - __uint_as_float(f.hi[i][e]));
        }
    }
}

// d += A(kt) B for one factor fragment (l0, l1): three TF32 products (the
// small cross terms first) or one.
template <int NT, int MODE>
__device__ __forceinline__ void mma_step(float (&d)[4], const Frag<NT, MODE>& a, int kt, float l0,
                                         float l1) {
    const unsigned h0 = f2tf32(l0), h1 = f2tf32(l1);
    if constexpr (MODE == 3) {
        const unsigned t0 = f2tf32(l0 - __uint_as_float(h0)), t1 = f2tf32(l1 - __uint_as_float(h1));
        mma_tf32(d, a.lo[kt][0], a.lo[kt][1], a.lo[kt][2], a.lo[kt][3], h0, h1);
        mma_tf32(d, a.hi[kt][0], a.hi[kt][1], a.hi[kt][2], a.hi[kt][3], t0, t1);
    }
    mma_tf32(d, a.hi[kt][0], a.hi[kt][1], a.hi[kt][2], a.hi[kt][3], h0, h1);
}

// out = X L for the panel X (16 shots x b, the transpose of L^T X): output
// tile nt sums the factor tiles (kt, nt), kt >= nt.
template <int NT, int MODE>
__device__ __forceinline__ void prod_l(const float* tl, const Frag<NT, MODE>& a, float (&out)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int o0 = 16 * t + g + 8 * (t >> 1);   // row 2t, column g of a tile
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = nt; kt < NT; ++kt) {
            const float* tile = tl + (kt * (kt + 1) / 2 + nt) * PTILE;
            mma_step<NT, MODE>(d, a, kt, tile[o0], tile[o0 + 8]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) out[nt][e] = d[e];
    }
}

// out = Z L^T (the transpose of L Z): output tile nt sums the factor tiles
// (nt, kt), kt <= nt.
template <int NT, int MODE>
__device__ __forceinline__ void prod_lt(const float* tl, const Frag<NT, MODE>& a, float (&out)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int o1 = 8 * g + 2 * t + 8 * (g >> 2);   // row g, columns 2t, 2t+1 of a tile
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt <= nt; ++kt) {
            const float2 l = *reinterpret_cast<const float2*>(tl + (nt * (nt + 1) / 2 + kt) * PTILE + o1);
            mma_step<NT, MODE>(d, a, kt, l.x, l.y);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) out[nt][e] = d[e];
    }
}

// y = L (L^T x) for the panel, in accumulator layout in and out.
template <int NT, int MODE>
__device__ __forceinline__ void factor_panel(const float* tl, const float (&x)[NT][4], float (&y)[NT][4]) {
    Frag<NT, MODE> f;
    split<NT, MODE>(x, f);
    float z[NT][4];
    prod_l<NT, MODE>(tl, f, z);
    split<NT, MODE>(z, f);
    prod_lt<NT, MODE>(tl, f, y);
}

// Panel of one level in accumulator layout: rows 8nt+2t, 8nt+2t+1, shots g
// and g+8; rows at or beyond b read as zero.
template <int NT>
__device__ __forceinline__ void ld_panel(const float* base, int b, float (&v)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int r0 = 8 * nt + 2 * t;
        float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
        if (r0 < b) a = *reinterpret_cast<const float2*>(base + r0 * 16 + 2 * g);
        if (r0 + 1 < b) c = *reinterpret_cast<const float2*>(base + (r0 + 1) * 16 + 2 * g);
        v[nt][0] = a.x; v[nt][2] = a.y; v[nt][1] = c.x; v[nt][3] = c.y;
    }
}

template <int NT>
__device__ __forceinline__ void st_panel(float* base, int b, const float (&v)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int r0 = 8 * nt + 2 * t;
        if (r0 < b) *reinterpret_cast<float2*>(base + r0 * 16 + 2 * g) = make_float2(v[nt][0], v[nt][2]);
        if (r0 + 1 < b) *reinterpret_cast<float2*>(base + (r0 + 1) * 16 + 2 * g) = make_float2(v[nt][1], v[nt][3]);
    }
}

// Receiver readout of one level: acc[pair][pos] += rho_{pair,j} . U_j for
// the pairs of the unit's subdomain (rows summed by lane, then a butterfly
// over t; the lanes t = 0 own the sums of shots g and g+8).
template <int NT>
__device__ __forceinline__ void readout_level(const PanelParams& p, int b, int j, int rp0, int nrp,
                                              const float (&u)[NT][4], float* acc) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int e = 0; e < nrp; ++e) {
        const int pr = p.sub_rp[rp0 + e];
        const float* row = p.rrows + p.rp_off[pr] + (long long)j * b;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int r0 = 8 * nt + 2 * t;
            const float a = r0 < b ? row[r0] : 0.f;
            const float c = r0 + 1 < b ? row[r0 + 1] : 0.f;
            s0 = fmaf(a, u[nt][0], s0);
            s1 = fmaf(a, u[nt][2], s1);
            s0 = fmaf(c, u[nt][1], s0);
            s1 = fmaf(c, u[nt][3], s1);
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if (t == 0) {
            acc[e * 16 + 2 * g] += s0;
            acc[e * 16 + 2 * g + 1] += s1;
        }
    }
}

// The same from rows staged in shared memory: rows[e * rstride + i] is row
// i of pair e's block at this level.
template <int NT>
__device__ __forceinline__ void readout_level_s(const float* rows, int rstride, int b, int nrp,
                                                const float (&u)[NT][4], float* acc) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int e = 0; e < nrp; ++e) {
        const float* row = rows + e * rstride;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int r0 = 8 * nt + 2 * t;
            const float a = r0 < b ? row[r0] : 0.f;
            const float c = r0 + 1 < b ? row[r0 + 1] : 0.f;
            s0 = fmaf(a, u[nt][0], s0);
            s1 = fmaf(a, u[nt][2], s1);
            s0 = fmaf(c, u[nt][1], s0);
            s1 = fmaf(c, u[nt][3], s1);
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if (t == 0) {
            acc[e * 16 + 2 * g] += s0;
            acc[e * 16 + 2 * g + 1] += s1;
        }
    }
}

// The unit's readout sums of sample n to the partial buffer, then cleared.
__device__ __forceinline__ void flush_readout(const PanelParams& p, int g, int n, int rp0, int nrp,
                                              float* acc) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int i = lane; i < nrp * 16; i += 32) {
        const int e = i >> 4, c = i & 15;
        const int pr = p.sub_rp[rp0 + e];
        p.partial[(((long long)g * (p.nsteps + 1) + n) * p.nrpairs + pr) * 16 + c] = acc[i];
        acc[i] = 0.f;
    }
    __syncwarp();
}

// Position in the stream of coefficient blocks shared by the consumer warps
// of a block: stage st, parity ph of its current use; a failed bounded wait
// marks the warp dead (it skips its remaining waits and arithmetic and
// leaves at the next device-wide barrier, which sees the error flag).
struct Ring {
    int st;
    unsigned ph;
    bool dead;
};

__device__ __forceinline__ const float* ring_take(Ring& r, const float* stages, int stage_elems,
                                                  unsigned long long* full, int* err,
                                                  unsigned long long timeout_ns) {
    if (!r.dead && !mbar_wait(full + r.st, r.ph, err, timeout_ns)) r.dead = true;
    return r.dead ? nullptr : stages + (size_t)r.st * stage_elems;
}

__device__ __forceinline__ const float* ring_take(Ring& r, const float* stages, int stage_elems,
                                                  unsigned long long* full, const PanelParams& p) {
    return ring_take(r, stages, stage_elems, full, p.err, p.timeout_ns);
}

__device__ __forceinline__ void ring_give(Ring& r, unsigned long long* empty, int nstage) {
    __syncwarp();
    if (!r.dead && (threadIdx.x & 31) == 0) mbar_arrive(empty + r.st);
    if (++r.st == nstage) { r.st = 0; r.ph ^= 1u; }
}

// Shared-memory panel slots of a warp: one level's b x 16 panel with a row
// stride of PROW floats (16 numbers + 4 of padding: rows 2t of the
// accumulator pattern then fall on distinct bank pairs for every t, so the
// float2 reads below are conflict free).
constexpr int PROW = 20;
constexpr int NSLOT = 5;           // U ring of 3, delta ring of 2
constexpr int RHO_STAGE_MAX = 8;   // receiver pairs per subdomain staged with the state

// Floats of a warp's shared-memory region: the state slots, two levels of
// staged receiver rows (when rpmax <= RHO_STAGE_MAX) and their offsets,
// rounded up to 128 bytes so that every warp's region (and the 16-byte
// copies into its slots) starts aligned.
__host__ __device__ inline long long warp_region_floats(int bmax, int rpmax) {
    const long long bpad = ((bmax + 7) / 8) * 8;
    const long long rho = rpmax <= RHO_STAGE_MAX ? rpmax : 0;
    const long long n = NSLOT * bpad * PROW + 2 * rho * bpad + 2 * rho;
    return (n + 31) / 32 * 32;
}

// Asynchronous copy (16-byte cp.async) of one level's panel (b rows of 16
// numbers, contiguous in global memory) into a slot.
__device__ __forceinline__ void stage_panel(float* slot, const float* src, int b) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < b * 4; i += 32) {
        const int r = i >> 2, c = i & 3;
        cp_async<16>(slot + r * PROW + 4 * c, src + r * 16 + 4 * c);
    }
}

template <int NT>
__device__ __forceinline__ void lds_panel(const float* slot, int b, float (&v)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int r0 = 8 * nt + 2 * t;
        float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
        if (r0 < b) a = *reinterpret_cast<const float2*>(slot + r0 * PROW + 2 * g);
        if (r0 + 1 < b) c = *reinterpret_cast<const float2*>(slot + (r0 + 1) * PROW + 2 * g);
        v[nt][0] = a.x; v[nt][2] = a.y; v[nt][1] = c.x; v[nt][3] = c.y;
    }
}

// Phase A of unit (group g, subdomain s) at step n (see the file comment).
// The warp stages the state it reads into its own slots one level ahead:
// copy group 0 holds U_0 and U_1, group j >= 1 holds U_{j+1} and delta_j,
// and group j+2 is issued as soon as level j has finished with the slots of
// U_j and delta_j, so the copies of the next levels run while this level's
// products do.  Only phi_{j-1} is carried from level to level in registers.
template <int NT, int MODE>
__device__ __noinline__ void unit_a(const PanelParams& p, int s, int g, int b, int k, int n, float* mail,
                       float* acc, float* slots, Ring& ring_io, const float* stages, int stage_elems,
                       unsigned long long* full, unsigned long long* empty) {
    Ring ring = ring_io;               // in registers for the level loop
    const int lane = threadIdx.x & 31, gg = lane >> 2;
    const long long so = ((long long)g * p.nstate + p.state_off[s]) * 16;
    float* U = p.U + so;
    float* D = p.dU + so;
    const long long sof = p.src_off[(long long)g * p.nsub + s];
    const float* src = sof >= 0 ? p.src + sof : nullptr;
    const float w0 = p.wavelet[(long long)(16 * g + gg) * p.nsteps + n];
    const float w1 = p.wavelet[(long long)(16 * g + gg + 8) * p.nsteps + n];
    const int rp0 = p.sub_rp_ptr[s], nrp = p.sub_rp_ptr[s + 1] - rp0;
    const float dt2 = p.dt2;
    const long long lb = (long long)b * 16;
    // fields the level loop needs, read once (the parameter block is not
    // in registers inside this function)
    int* const err = p.err;
    const unsigned long long tmo = p.timeout_ns;
    const int nstage = p.nstage;
    const int bpad = ((p.bmax + 7) / 8) * 8;
    const int ss = bpad * PROW;                            // floats per slot
    float* Us = slots;                                     // U slots 0..2
    float* Ds = slots + 3 * ss;                            // delta slots 0..1
    // receiver rows of levels j (parity j & 1), with the pairs' row offsets
    const bool rho_st = p.rpmax <= RHO_STAGE_MAX && nrp > 0;
    float* Rs = slots + NSLOT * ss;
    const int rsz = p.rpmax * bpad;
    long long* rpb = reinterpret_cast<long long*>(Rs + 2 * rsz);
    const float* rrows = p.rrows;
    if (rho_st) {
        for (int e = lane; e < nrp; e += 32) rpb[e] = p.rp_off[p.sub_rp[rp0 + e]];
        __syncwarp();
    }
    // group j of copies (see above; with receivers also their rows of
    // level j); an empty group is committed too, so the group count stays
    // the same in every lane
    auto issue = [&](int j) {
        if (j == 0) {
            stage_panel(Us, U, b);
            if (k > 1) stage_panel(Us + ss, U + lb, b);
        } else if (j < k) {
            if (j + 1 < k) stage_panel(Us + ((j + 1) % 3) * ss, U + (j + 1) * lb, b);
            stage_panel(Ds + (j & 1) * ss, D + j * lb, b);
        }
        if (rho_st && j < k)
            for (int e = 0; e < nrp; ++e)
                for (int i = lane; i < b; i += 32)
                    cp_async<4>(Rs + (j & 1) * rsz + e * bpad + i, rrows + rpb[e] + (long long)j * b + i);
        cp_async_commit();
    };
    __syncwarp();
    issue(0);
    issue(1);
    float phiprev[NT][4];
    for (int j = 0; j < k; ++j) {
        cp_async_wait<1>();
        __syncwarp();
        const float* Uj = Us + (j % 3) * ss;
        const float* Uj1 = Us + ((j + 1) % 3) * ss;
        const float* Dj = Ds + (j & 1) * ss;
        float x[NT][4], y[NT][4];
        // Delta_j = U_{j+1} - U_j (U_k = 0), and the readout of U_j^n
        lds_panel<NT>(Uj, b, y);
        if (rho_st) readout_level_s<NT>(Rs + (j & 1) * rsz, bpad, b, nrp, y, acc);
        else if (nrp > 0) readout_level<NT>(p, b, j, rp0, nrp, y, acc);
        if (j + 1 < k) {
            lds_panel<NT>(Uj1, b, x);
        } else {
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) x[i][e] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) x[i][e] -= y[i][e];
        const float* tl = ring_take(ring, stages, stage_elems, full, err, tmo);
        if (tl) factor_panel<NT, MODE>(tl, x, y);     // y = phi_j
        ring_give(ring, empty, nstage);
        // x = p_j f(t_n)
        if (src) {
            ld_panel<NT>(src + j * lb, b, x);
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                x[i][0] *= w0; x[i][1] *= w0; x[i][2] *= w1; x[i][3] *= w1;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) x[i][e] = 0.f;
        }
        if (j == 0) {
            // (2.1) face data [phi_0 + p_0 f]
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    phiprev[i][e] = y[i][e];
                    x[i][e] += y[i][e];
                }
            st_panel<NT>(mail + ((long long)g * p.nmail + p.mail_off[s]) * 16, b, x);
        } else {
            // psi_j = phi_j - phi_{j-1} + p_j f
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    x[i][e] = (y[i][e] - phiprev[i][e]) + x[i][e];
                    phiprev[i][e] = y[i][e];
                }
            tl = ring_take(ring, stages, stage_elems, full, err, tmo);
            if (tl) factor_panel<NT, MODE>(tl, x, y);     // y = a_j
            ring_give(ring, empty, nstage);
            if (tl) {
                // (2.2) increment and state update, Eq. (19)
                lds_panel<NT>(Dj, b, x);
#pragma unroll
                for (int i = 0; i < NT; ++i)
#pragma unroll
                    for (int e = 0; e < 4; ++e) x[i][e] = fmaf(dt2, y[i][e], x[i][e]);
                st_panel<NT>(D + j * lb, b, x);
                lds_panel<NT>(Uj, b, y);
#pragma unroll
                for (int i = 0; i < NT; ++i)
#pragma unroll
                    for (int e = 0; e < 4; ++e) y[i][e] += x[i][e];
                st_panel<NT>(U + j * lb, b, y);
            }
        }
        // the slots of U_j and delta_j are free: stage two levels ahead
        __syncwarp();
        issue(j + 2);
    }
    cp_async_wait<0>();
    __syncwarp();
    ring_io = ring;
    if (nrp > 0) flush_readout(p, g, n, rp0, nrp, acc);
}

// Readout of the final sample (U after the last step).
template <int NT>
__device__ void unit_final_readout(const PanelParams& p, int s, int g, int b, int k, float* acc) {
    const int rp0 = p.sub_rp_ptr[s], nrp = p.sub_rp_ptr[s + 1] - rp0;
    if (nrp == 0) return;
    const float* U = p.U + ((long long)g * p.nstate + p.state_off[s]) * 16;
    for (int j = 0; j < k; ++j) {
        float u[NT][4];
        ld_panel<NT>(U + (long long)j * b * 16, b, u);
        readout_level<NT>(p, b, j, rp0, nrp, u, acc);
    }
    flush_readout(p, g, p.nsteps, rp0, nrp, acc);
}

// Phase B of unit (g, s): face sums of both sides (lower subdomain first, so
// both sides form the same sum), a_f = H_f sum (Eq. 18), level-0 update.
__device__ void unit_b(const PanelParams& p, int s, int g, int b, int n, const float* mail, float* scr) {
    const int lane = threadIdx.x & 31;
    const long long mrow = p.mail_off[s];
    const long long mg = (long long)g * p.nmail;
    for (int i = lane; i < b * 16; i += 32) {
        const int r = i >> 4, c = i & 15;
        const int4 e = p.frow[mrow + r];
        float v = mail[(mg + mrow + r) * 16 + c];
        if (e.x >= 0) {
            const float o = mail[(mg + e.x) * 16 + c];
            v = (e.z >> 16) ? o + v : v + o;
        }
        scr[i] = v;
    }
    __syncwarp();
    const long long so = ((long long)g * p.nstate + p.state_off[s]) * 16;
    for (int i = lane; i < b * 16; i += 32) {
        const int r = i >> 4, c = i & 15;
        const int4 e = p.frow[mrow + r];
        const int m = e.z & 0xffff;
        const float* H = p.H + e.y;
        const float* v = scr + e.w * 16 + c;
        float a = 0.f;
        for (int cc = 0; cc < m; ++cc) a = fmaf(H[cc * m], v[cc * 16], a);
        const float d = fmaf(p.dt2, a, p.dU[so + i]);
        p.dU[so + i] = d;
        const float un = p.U[so + i] + d;
        p.U[so + i] = un;
        if (!(fabsf(un) < 1e30f)) {
            // instability sentinel: every block leaves at the next barrier
            if (p.ustep) atomicMin(p.ustep, n);
            atomicCAS(p.err, 0, (int)SFM_ERR_UNSTABLE);
        }
    }
    __syncwarp();
}

template <int MODE>
__device__ __forceinline__ void unit_a_any(int nt, const PanelParams& p, int s, int g, int b, int k,
                                           int n, float* mail, float* acc, float* slots, Ring& ring,
                                           const float* stages, int stage_elems,
                                           unsigned long long* full, unsigned long long* empty) {
    switch (nt) {
        case 1: unit_a<1, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 2: unit_a<2, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 3: unit_a<3, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 4: unit_a<4, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 5: unit_a<5, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 6: unit_a<6, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 7: unit_a<7, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        default: unit_a<8, MODE>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
    }
}

__device__ __forceinline__ void final_readout_any(int nt, const PanelParams& p, int s, int g, int b,
                                                  int k, float* acc) {
    switch (nt) {
        case 1: unit_final_readout<1>(p, s, g, b, k, acc); break;
        case 2: unit_final_readout<2>(p, s, g, b, k, acc); break;
        case 3: unit_final_readout<3>(p, s, g, b, k, acc); break;
        case 4: unit_final_readout<4>(p, s, g, b, k, acc); break;
        case 5: unit_final_readout<5>(p, s, g, b, k, acc); break;
        case 6: unit_final_readout<6>(p, s, g, b, k, acc); break;
        case 7: unit_final_readout<7>(p, s, g, b, k, acc); break;
        default: unit_final_readout<8>(p, s, g, b, k, acc); break;
    }
}

// The persistent multi-shot stepping kernel: p.ncw consumer warps (one
// 16-shot group each) and one producer warp whose lane 0 streams every task's
// factors, in the order Gamma_0, Gamma_1, Gammahat_1, ..., Gamma_{k-1},
// Gammahat_{k-1}, with bulk asynchronous copies through a ring of p.nstage
// shared-memory stages; all consumer warps read every stage (a task's warps
// work on the same subdomain), warps without a group pass over it.
template <int MODE>
__global__ void __launch_bounds__(PANEL_BLOCK_MAX) panel_kernel(const __grid_constant__ PanelParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ncw = p.ncw, nct = ncw * 32, nstage = p.nstage;
    const int stage_elems = (int)(tri_tiles(p.bmax) * PTILE);
    const int bpad = ((p.bmax + 7) / 8) * 8;
    float* stages = reinterpret_cast<float*>(smem_raw);
    const long long wreg = warp_region_floats(p.bmax, p.rpmax);
    float* slot_all = stages + (size_t)nstage * stage_elems;         // ncw x wreg
    float* acc_all = slot_all + (size_t)ncw * wreg;                 // ncw x rpmax*16
    unsigned long long* full = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(acc_all + (size_t)ncw * p.rpmax * 16) + 15) & ~(uintptr_t)15);
    unsigned long long* empty = full + nstage;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tk0 = p.task_ptr[blockIdx.x], tk1 = p.task_ptr[blockIdx.x + 1];
    if (threadIdx.x == 0) {
        for (int i = 0; i < nstage; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, ncw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < ncw * p.rpmax * 16; i += blockDim.x) acc_all[i] = 0.f;
    __syncthreads();

    if (warp == ncw) {
        // ------------------------------ producer ------------------------------
        if (lane != 0) return;
        long long gcount = 0;
        int st = 0;
        unsigned ph = 0;
        bool ok = true;
        for (int n = 0; n < p.nsteps && ok; ++n) {
            for (int tk = tk0; tk < tk1 && ok; ++tk) {
                const int4 T = p.task[tk];
                const int b = T.w & 255, k = T.w >> 8;
                const long long ltile = tri_tiles(b) * PTILE;
                const unsigned bytes = (unsigned)(ltile * sizeof(float));
                const long long base = p.coef_off[T.x];
                for (int m = 0; m < 2 * k - 1; ++m, ++gcount) {
                    if (gcount >= nstage && !mbar_wait(empty + st, ph ^ 1u, p.err, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    // stream block m: Gamma_0 (m = 0), Gamma_j (m = 2j-1), Gammahat_j
                    // (m = 2j), stored level-major as [Gamma_j][Gammahat_j]
                    const long long off = base + (m == 0 ? 0 : (long long)(m + 1)) * ltile;
                    mbar_expect_tx(full + st, bytes);
                    bulk_g2s(stages + (size_t)st * stage_elems, p.coef + off, bytes, full + st);
                    if (++st == nstage) { st = 0; ph ^= 1u; }
                }
            }
        }
        // never leave with copies in flight
        for (long long h = (gcount > nstage ? gcount - nstage : 0); h < gcount; ++h)
            mbar_wait(full + (int)(h % nstage), (unsigned)((h / nstage) & 1), p.err, p.timeout_ns);
        return;
    }

    // ------------------------------- consumers --------------------------------
    float* slots = slot_all + (size_t)warp * wreg;
    float* scr = slots;                  // phase B's face sums reuse the first slot
    float* acc = acc_all + (size_t)warp * p.rpmax * 16;
    Ring ring{0, 0u, false};
    for (int n = 0; n < p.nsteps; ++n) {
        float* mail = (n & 1) ? p.mail1 : p.mail0;
        for (int tk = tk0; tk < tk1; ++tk) {
            const int4 T = p.task[tk];
            const int s = T.x, b = T.w & 255, k = T.w >> 8;
            if (warp < T.z) {
                unit_a_any<MODE>((b + 7) >> 3, p, s, T.y + warp, b, k, n, mail, acc, slots, ring, stages,
                                 stage_elems, full, empty);
            } else {
                for (int m = 0; m < 2 * k - 1; ++m) {
                    ring_take(ring, stages, stage_elems, full, p);
                    ring_give(ring, empty, nstage);
                }
            }
        }
        grid_arrive(p.bar, p.skip_arrive, nct);
        if (!grid_wait(p.bar, (unsigned)(n + 1) * gridDim.x, p.err, p.timeout_ns, nct)) return;
        for (int tk = tk0; tk < tk1; ++tk) {
            const int4 T = p.task[tk];
            if (warp < T.z) unit_b(p, T.x, T.y + warp, T.w & 255, n, mail, scr);
        }
    }
    for (int tk = tk0; tk < tk1; ++tk) {
        const int4 T = p.task[tk];
        const int b = T.w & 255;
        if (warp < T.z) final_readout_any((b + 7) >> 3, p, T.x, T.y + warp, b, T.w >> 8, acc);
    }
}

size_t panel_smem_bytes(int ncw, int nstage, int bmax, int rpmax) {
    const size_t bpad = (size_t)((bmax + 7) / 8) * 8;
    (void)bpad;
    size_t bytes = sizeof(float) * ((size_t)nstage * tri_tiles(bmax) * PTILE +
                                    (size_t)ncw * warp_region_floats(bmax, rpmax) + (size_t)ncw * rpmax * 16);
    bytes = (bytes + 15) & ~(size_t)15;
    return bytes + 2 * (size_t)nstage * sizeof(unsigned long long);
}

template <int MODE>
static int panel_max_grid_t(int ncw, size_t smem, int* grid_out) {
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(panel_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel<MODE>, (ncw + 1) * 32, smem);
    if (per_sm < 1) return -1;
    *grid_out = per_sm * nsm;
    return 0;
}

int panel_max_grid(int mode, int ncw, size_t smem, int* grid_out) {
    return mode == 3 ? panel_max_grid_t<3>(ncw, smem, grid_out) : panel_max_grid_t<1>(ncw, smem, grid_out);
}

template <int MODE>
static cudaError_t launch_panel_t(const PanelParams& p, int grid, cudaStream_t st) {
    const size_t smem = panel_smem_bytes(p.ncw, p.nstage, p.bmax, p.rpmax);
    cudaError_t e = cudaFuncSetAttribute(panel_kernel<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PanelParams pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((void*)panel_kernel<MODE>, dim3(grid), dim3((p.ncw + 1) * 32),
                                       args, smem, st);
}

cudaError_t launch_panel(int mode, const PanelParams& p, int grid, cudaStream_t st) {
    return mode == 3 ? launch_panel_t<3>(p, grid, st) : launch_panel_t<1>(p, grid, st);
}

// Tasks (subdomain, chunk of at most ncw 16-shot groups), longest first,
// each to the block with the least estimated cost so far (a task's cost:
// its k levels of four factor products of nt(nt+1)/2 tiles each, plus a
// fixed part for its face work and stream start).
void build_panel_tasks(int nsub, int ngroups, const int* k_sub, const int* b_sub, int ncw,
                       int grid, std::vector<int>& ptr, std::vector<int4>& tasks) {
    struct T {
        int4 t;
        double cost;
    };
    std::vector<T> all;
    for (int s = 0; s < nsub; ++s) {
        const int nt = (b_sub[s] + 7) / 8;
        const double cost = (double)k_sub[s] * (2.0 * nt * (nt + 1)) + 2.0 * nt * nt + 8.0;
        for (int g0 = 0; g0 < ngroups; g0 += ncw)
            all.push_back({make_int4(s, g0, std::min(ncw, ngroups - g0), b_sub[s] | (k_sub[s] << 8)), cost});
    }
    std::stable_sort(all.begin(), all.end(), [](const T& a, const T& b) { return a.cost > b.cost; });
    std::vector<std::vector<int4>> per(grid);
    std::vector<double> load(grid, 0.0);
    for (const T& t : all) {
        int best = 0;
        for (int c = 1; c < grid; ++c)
            if (load[c] < load[best]) best = c;
        load[best] += t.cost;
        per[best].push_back(t.t);
    }
    ptr.assign(grid + 1, 0);
    tasks.clear();
    for (int c = 0; c < grid; ++c) {
        // in subdomain order inside a block (a fixed, shape-independent walk)
        std::sort(per[c].begin(), per[c].end(),
                  [](const int4& a, const int4& b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
        for (const int4& t : per[c]) tasks.push_back(t);
        ptr[c + 1] = (int)tasks.size();
    }
}

__global__ void pad_tiles_kernel(const float* in, float* out, long long ntiles) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ntiles * PTILE;
         i += (long long)gridDim.x * blockDim.x) {
        const long long tile = i / PTILE;
        const int e = (int)(i - tile * PTILE);
        // e = r*8 + c + 8*(r >> 2): rows 0..3 at 0..31, 32..39 unused, rows 4..7 at 40..71
        float v = 0.f;
        if (e < 32) v = in[tile * 64 + e];
        else if (e >= 40) v = in[tile * 64 + (e - 8)];
        out[i] = v;
    }
}

cudaError_t launch_pad_tiles(const float* in, float* out, long long ntiles, cudaStream_t st) {
    const long long n = ntiles * PTILE;
    const int grid = (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 8192);
    pad_tiles_kernel<<<grid, 256, 0, st>>>(in, out, ntiles);
    return cudaGetLastError();
}

__device__ __forceinline__ int panel_pos(int c) { return 2 * (c & 7) + (c >> 3); }

__global__ void to_panel_kernel(const double* in, float* out, int nshots, long long n, int ngroups) {
    const long long total = (long long)ngroups * n * 16;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int pos = (int)(i & 15);
        const long long ge = i >> 4;
        const int g = (int)(ge / n);
        const long long e = ge - (long long)g * n;
        const int c = (pos >> 1) + 8 * (pos & 1);
        const int q = 16 * g + c;
        out[i] = q < nshots ? (float)in[(long long)q * n + e] : 0.f;
    }
}

cudaError_t launch_to_panel(const double* in, float* out, int nshots, long long n, cudaStream_t st) {
    const int ngroups = (nshots + 15) / 16;
    const long long total = (long long)ngroups * n * 16;
    const int grid = (int)std::min<long long>(std::max<long long>((total + 255) / 256, 1), 8192);
    to_panel_kernel<<<grid, 256, 0, st>>>(in, out, nshots, n, ngroups);
    return cudaGetLastError();
}

__global__ void from_panel_kernel(const float* in, double* out, int nshots, long long n) {
    const long long total = (long long)nshots * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / n);
        const long long e = i - (long long)q * n;
        out[i] = (double)in[(((long long)(q >> 4)) * n + e) * 16 + panel_pos(q & 15)];
    }
}

cudaError_t launch_from_panel(const float* in, double* out, int nshots, long long n, cudaStream_t st) {
    const long long total = (long long)nshots * n;
    const int grid = (int)std::min<long long>(std::max<long long>((total + 255) / 256, 1), 8192);
    from_panel_kernel<<<grid, 256, 0, st>>>(in, out, nshots, n);
    return cudaGetLastError();
}

__global__ void src_panels_kernel(const double* rows, const long long* off64, const long long* dst,
                                  const int* len, float* out) {
    const int i = blockIdx.x;
    const long long d = dst[i], base = d - (d & 15);
    const int pos = (int)(d & 15);
    for (int e = threadIdx.x; e < len[i]; e += blockDim.x)
        out[base + (long long)e * 16 + pos] = (float)rows[off64[i] + e];
}

cudaError_t launch_src_panels(const double* rows, const long long* off64, const long long* dst,
                              const int* len, int npairs, float* out, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    src_panels_kernel<<<npairs, 128, 0, st>>>(rows, off64, dst, len, out);
    return cudaGetLastError();
}

__global__ void panel_traces_kernel(const float* partial, const int* rec_ptr, const int* rec_pairs,
                                    int nshots, int nsteps, int nrec, int nrpairs, double* traces,
                                    int* bad) {
    const long long total = (long long)nshots * nrec * (nsteps + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i % (nsteps + 1));
        const long long qr = i / (nsteps + 1);
        const int r = (int)(qr % nrec), q = (int)(qr / nrec);
        const long long row = ((long long)(q >> 4) * (nsteps + 1) + n) * nrpairs;
        const int pos = panel_pos(q & 15);
        double acc = 0.0;
        for (int e = rec_ptr[r]; e < rec_ptr[r + 1]; ++e)
            acc += (double)partial[(row + rec_pairs[e]) * 16 + pos];
        traces[i] = acc;
        if (!isfinite(acc)) atomicExch(bad, 1);
    }
}

cudaError_t launch_panel_traces(const float* partial, const int* rec_ptr, const int* rec_pairs,
                                int nshots, int nsteps, int nrec, int nrpairs, double* traces,
                                int* bad, cudaStream_t st) {
    const long long total = (long long)nshots * nrec * (nsteps + 1);
    const int grid = (int)std::min<long long>(std::max<long long>((total + 255) / 256, 1), 4096);
    panel_traces_kernel<<<grid, 256, 0, st>>>(partial, rec_ptr, rec_pairs, nshots, nsteps, nrec,
                                              nrpairs, traces, bad);
    return cudaGetLastError();
}

}  // namespace sfm
