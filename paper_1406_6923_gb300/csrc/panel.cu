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
// phi_{j-1} in the accumulator layout (4 nt numbers a lane), rounded up to
// 128 bytes so that every warp's region (and the 16-byte copies into its
// slots) starts aligned.
__host__ __device__ inline long long warp_region_floats(int bmax, int rpmax) {
    const long long bpad = ((bmax + 7) / 8) * 8;
    const long long rho = rpmax <= RHO_STAGE_MAX ? rpmax : 0;
    const long long n = NSLOT * bpad * PROW + 2 * rho * bpad + 2 * rho + 16 * bpad;
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
    // shared-memory pointers re-derived from the kernel's dynamic shared
    // memory (whose base is the ring): through the call they arrive as
    // generic addresses, and loads through generic addresses wait on the
    // long scoreboard; derived from the __shared__ array they compile to
    // shared-memory loads
    extern __shared__ __align__(128) unsigned char smem_raw[];
    {
        float* const sm0 = reinterpret_cast<float*>(smem_raw);
        slots = sm0 + (slots - stages);
        acc = sm0 + (acc - stages);
        stages = sm0;
    }
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
    // phi_{j-1}, lane-private in shared memory (entry (i, e) of this lane at
    // (i*4 + e)*32 + lane): a register copy would spill
    const long long rho_n = p.rpmax <= RHO_STAGE_MAX ? p.rpmax : 0;
    float* const phiprev = slots + NSLOT * ss + 2 * rho_n * bpad + 2 * rho_n;
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
                    phiprev[(i * 4 + e) * 32 + lane] = y[i][e];
                    x[i][e] += y[i][e];
                }
            st_panel<NT>(mail + ((long long)g * p.nmail + p.mail_off[s]) * 16, b, x);
        } else {
            // psi_j = phi_j - phi_{j-1} + p_j f
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float* pp = phiprev + (i * 4 + e) * 32 + lane;
                    x[i][e] = (y[i][e] - *pp) + x[i][e];
                    *pp = y[i][e];
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

// ---------------------------------------------------------------------------
// Two-float panels (SFM_FP32X2P): the stepping above with the state, the face
// data, H_f and the S-fraction blocks in two-float form (x = hi + lo, two FP32
// words, as SFM_FP32X2) and the block products on the CUDA cores.  Every
// streamed block Gamma (symmetric, kept as the upper triangle of 8x8 tiles) is
// applied to a 16-shot panel as 16 compensated dot products per row: per term
// the FMA two-product of the head words and Knuth's two-sum into the running
// head, with the rounding errors and the two cross terms (head x tail) summed
// beside it (Ogita, Rump and Oishi's Dot2 arrangement).  Deep ROMs whose
// blocks are too ill-conditioned for FP32 coefficients or an FP32 state step
// at SFM_FP32X2's accuracy, with each block read once for 16 shots.
//
// Layout (floats):
//   state panel of (group g, subdomain s, level j): b rows of 16 shots x
//   (hi, lo); row i of shot c at (j*b + i)*32 + 2c (+1 for lo); groups at
//   g * nstate * 32, subdomain s at state_off[s] * 32 inside its group; face
//   data likewise over the level-0 rows (mail_off);
//   block tiles: tile (I, J) (J >= I) of the upper triangle at
//   I*nt - I(I-1)/2 + (J - I), 144 floats per tile: row r, column c at
//   2*(9r + c) (+1 for lo), column 8 zero (the padding column makes both the
//   row reads and the transposed reads below free of bank conflicts); per
//   level Gamma_j then Gammahat_j, offsets coef_off (floats);
//   H_f: two-float pairs at 2 * H offset.
// Lane (q, a) = (lane >> 3, lane & 7) of a warp owns shots 4q..4q+3 of rows
// 8R + a (R < nt) of its unit.
constexpr int P2TILE = 144;   // floats per padded two-float tile
constexpr int P2ROW = 36;     // floats per staged panel row (32 + 4 of padding)

// Compensated a += g x for two-float g = (gh, gl), x = (xh, xl): the head
// product's rounding error (FMA) and the two-sum's error go to e with the
// cross terms; s + e is the running sum.
__device__ __forceinline__ void x2_fma(float& s, float& e, float gh, float gl, float xh, float xl) {
    const float pr = __fmul_rn(gh, xh);
    const float pe = fmaf(gh, xh, -pr);
    const float t = __fadd_rn(s, pr);
    const float z = __fsub_rn(t, s);
    const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(pr, z));
    s = t;
    e = __fadd_rn(e, __fadd_rn(se, pe));
    e = fmaf(gh, xl, e);
    e = fmaf(gl, xh, e);
}

// (s, e) -> normalised two-float (hi, lo)
__device__ __forceinline__ df x2_norm(float s, float e) { return quick_two_sum(s, e); }

__device__ __forceinline__ df x2_neg(df a) { return {-a.hi, -a.lo}; }

// y[R][c] = sum_i G[8R + a][i] X[i][4q + c] for the symmetric block in `tl`
// (nt = NT tiles a side, zero beyond b) and the staged panel X (rows of
// P2ROW floats, zero from b to 8 NT), as unnormalised (s, e) pairs.
template <int NT>
__device__ __forceinline__ void sym2_apply(const float* tl, const float* X, float (&s)[NT][4], float (&e)[NT][4]) {
    const int lane = threadIdx.x & 31, q = lane >> 3, a = lane & 7;
#pragma unroll
    for (int R = 0; R < NT; ++R)
#pragma unroll
        for (int c = 0; c < 4; ++c) s[R][c] = e[R][c] = 0.f;
#pragma unroll
    for (int K = 0; K < NT; ++K) {
#pragma unroll 1
        for (int bb = 0; bb < 8; ++bb) {
            const float* xr = X + (8 * K + bb) * P2ROW + 8 * q;
            const float* trow = tl + 2 * (9 * a + bb);   // element (a, bb) of a tile
            const float* tcol = tl + 2 * (9 * bb + a);   // element (bb, a)
            const float4 x0 = *reinterpret_cast<const float4*>(xr);
            const float4 x1 = *reinterpret_cast<const float4*>(xr + 4);
#pragma unroll
            for (int R = 0; R < NT; ++R) {
                // G[8R + a][8K + bb]: tile (R, K) element (a, bb) at or above
                // the diagonal, else tile (K, R) element (bb, a)
                const int tix = R <= K ? R * NT - R * (R - 1) / 2 + (K - R) : K * NT - K * (K - 1) / 2 + (R - K);
                const float2 g = *reinterpret_cast<const float2*>((R <= K ? trow : tcol) + tix * P2TILE);
                x2_fma(s[R][0], e[R][0], g.x, g.y, x0.x, x0.y);
                x2_fma(s[R][1], e[R][1], g.x, g.y, x0.z, x0.w);
                x2_fma(s[R][2], e[R][2], g.x, g.y, x1.x, x1.y);
                x2_fma(s[R][3], e[R][3], g.x, g.y, x1.z, x1.w);
            }
        }
    }
}

// Two-float rows of a panel in global memory (row stride 32 floats) at the
// lane's positions: shots 4q..4q+3 of row r as two float4 (hi, lo pairs).
__device__ __forceinline__ void ldg2_row(const float* base, int r, int q, float4& u0, float4& u1) {
    u0 = *reinterpret_cast<const float4*>(base + r * 32 + 8 * q);
    u1 = *reinterpret_cast<const float4*>(base + r * 32 + 8 * q + 4);
}

__device__ __forceinline__ void stg2_row(float* base, int r, int q, const df (&v)[4]) {
    *reinterpret_cast<float4*>(base + r * 32 + 8 * q) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    *reinterpret_cast<float4*>(base + r * 32 + 8 * q + 4) = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
}

__device__ __forceinline__ void unpack4(const float4& u0, const float4& u1, df (&v)[4]) {
    v[0] = {u0.x, u0.y}; v[1] = {u0.z, u0.w}; v[2] = {u1.x, u1.y}; v[3] = {u1.z, u1.w};
}

// Merge of two unnormalised compensated sums (s1 + e1) + (s2 + e2).
__device__ __forceinline__ void x2_merge(float& s, float& e, float s2, float e2) {
    const df t = two_sum(s, s2);
    s = t.hi;
    e = __fadd_rn(__fadd_rn(e, e2), t.lo);
}

// Readout of level j of the state at U (global, the unit's panel) with the
// two-float receiver rows: compensated sums over the lane's rows, merged
// across the eight row lanes, added to acc[pair][pos(c)] as (hi, lo).  The
// lane's state values are loaded once for all the unit's pairs.
template <int NT>
__device__ __forceinline__ void readout_level2(const PanelParams& p, const float* U, int b, int j, int rp0,
                                               int nrp, float* acc) {
    const int lane = threadIdx.x & 31, q = lane >> 3, a = lane & 7;
    const float* Uj = U + (long long)j * b * 32;
    float4 u0[NT], u1[NT];
#pragma unroll
    for (int R = 0; R < NT; ++R) {
        const int r = 8 * R + a;
        u0[R] = u1[R] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < b) ldg2_row(Uj, r, q, u0[R], u1[R]);
    }
    for (int e = 0; e < nrp; ++e) {
        const int pr = p.sub_rp[rp0 + e];
        const float* row = p.rrows + 2 * (p.rp_off[pr] + (long long)j * b);
        float ts[4] = {0.f, 0.f, 0.f, 0.f}, te[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int R = 0; R < NT; ++R) {
            const int r = 8 * R + a;
            if (r < b) {
                const float2 w = *reinterpret_cast<const float2*>(row + 2 * r);
                x2_fma(ts[0], te[0], w.x, w.y, u0[R].x, u0[R].y);
                x2_fma(ts[1], te[1], w.x, w.y, u0[R].z, u0[R].w);
                x2_fma(ts[2], te[2], w.x, w.y, u1[R].x, u1[R].y);
                x2_fma(ts[3], te[3], w.x, w.y, u1[R].z, u1[R].w);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, ts[c], o);
                const float e2 = __shfl_xor_sync(0xffffffffu, te[c], o);
                x2_merge(ts[c], te[c], s2, e2);
            }
        }
        if (a == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int sh = 4 * q + c;
                float2* ap = reinterpret_cast<float2*>(acc) + e * 16 + 2 * (sh & 7) + (sh >> 3);
                const df sum = df_add(df{ap->x, ap->y}, x2_norm(ts[c], te[c]));
                *ap = make_float2(sum.hi, sum.lo);
            }
        }
    }
    __syncwarp();
}

// The unit's readout sums of sample n (two-float) to the partial buffer
// ([g][n][pair][pos] pairs), then cleared.
__device__ __forceinline__ void flush_readout2(const PanelParams& p, int g, int n, int rp0, int nrp, float* acc) {
    const int lane = threadIdx.x & 31;
    float2* a2 = reinterpret_cast<float2*>(acc);
    float2* part = reinterpret_cast<float2*>(p.partial);
    __syncwarp();
    for (int i = lane; i < nrp * 16; i += 32) {
        const int e = i >> 4, c = i & 15;
        const int pr = p.sub_rp[rp0 + e];
        part[(((long long)g * (p.nsteps + 1) + n) * p.nrpairs + pr) * 16 + c] = a2[i];
        a2[i] = make_float2(0.f, 0.f);
    }
    __syncwarp();
}

// Y = G X for the staged panel X, normalised two-float, written to shared
// memory in the lane's own layout (entry (R, c) of lane l at (R*4 + c)*32 + l).
template <int NT>
__device__ __forceinline__ void sym2_to(const float* tl, const float* X, float2* Y) {
    float ys[NT][4], ye[NT][4];
    sym2_apply<NT>(tl, X, ys, ye);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int R = 0; R < NT; ++R)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const df v = x2_norm(ys[R][c], ye[R][c]);
            Y[(R * 4 + c) * 32 + lane] = make_float2(v.hi, v.lo);
        }
}

// Phase A of unit (g, s) at step n in two-float form (see unit_a).  The
// warp's shared memory holds the product input X (Delta_j, then psi_j, a
// panel of P2ROW-float rows) and two product outputs in the lane's own
// layout, used in turn: level j writes phi_j into one while the other holds
// phi_{j-1}, then a_j over phi_{j-1}.  The state and the increments are read
// from global memory at the lane's positions.
template <int NT>
__device__ __forceinline__ void unit_a2(const PanelParams& p, int s, int g, int b, int k, int n, float* mail,
                                        float* acc, float* slots, Ring& ring, const float* stages,
                                        int stage_elems, unsigned long long* full, unsigned long long* empty) {
    const int lane = threadIdx.x & 31, q = lane >> 3, a = lane & 7;
    const long long so = ((long long)g * p.nstate + p.state_off[s]) * 32;
    float* U = p.U + so;
    float* D = p.dU + so;
    const long long sof = p.src_off[(long long)g * p.nsub + s];
    const float* src = sof >= 0 ? p.src + sof : nullptr;
    float w[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) w[c] = p.wavelet[(long long)(16 * g + 4 * q + c) * p.nsteps + n];
    const int rp0 = p.sub_rp_ptr[s], nrp = p.sub_rp_ptr[s + 1] - rp0;
    const df dt2 = {p.dt2, p.dt2lo};
    const int bpad = ((p.bmax + 7) / 8) * 8;
    float* X = slots;
    float2* Y0 = reinterpret_cast<float2*>(slots + bpad * P2ROW);
    float2* Y1 = Y0 + bpad * 16;
    float* Mq = mail + ((long long)g * p.nmail + p.mail_off[s]) * 32;
    const long long lb = (long long)b * 32;
    for (int j = 0; j < k; ++j) {
        float2* cur = (j & 1) ? Y1 : Y0;     // phi_j, then (next level) phi_{j-1}
        float2* prv = (j & 1) ? Y0 : Y1;     // phi_{j-1}, then a_j
        const float* Uj = U + j * lb;
        if (nrp > 0) readout_level2<NT>(p, U, b, j, rp0, nrp, acc);
        // X = Delta_j = U_{j+1} - U_j (U_k = 0; rows from b on zero)
        __syncwarp();
#pragma unroll
        for (int R = 0; R < NT; ++R) {
            const int r = 8 * R + a;
            float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
            if (r < b) {
                float4 u0, u1, v0 = x0, v1 = x0;
                ldg2_row(Uj, r, q, u0, u1);
                if (j + 1 < k) ldg2_row(Uj + lb, r, q, v0, v1);
                df uu[4], vv[4];
                unpack4(u0, u1, uu);
                unpack4(v0, v1, vv);
#pragma unroll
                for (int c = 0; c < 4; ++c) vv[c] = df_add(vv[c], x2_neg(uu[c]));
                x0 = make_float4(vv[0].hi, vv[0].lo, vv[1].hi, vv[1].lo);
                x1 = make_float4(vv[2].hi, vv[2].lo, vv[3].hi, vv[3].lo);
            }
            *reinterpret_cast<float4*>(X + r * P2ROW + 8 * q) = x0;
            *reinterpret_cast<float4*>(X + r * P2ROW + 8 * q + 4) = x1;
        }
        __syncwarp();
        const float* tl = ring_take(ring, stages, stage_elems, full, p);
        if (tl) sym2_to<NT>(tl, X, cur);                       // phi_j
        ring_give(ring, empty, p.nstage);
        if (!tl) continue;
        __syncwarp();                                           // every lane is done with X
        // psi_j = phi_j - phi_{j-1} + p_j f into X (j >= 1), or the face data
        // phi_0 + p_0 f (j = 0)
#pragma unroll
        for (int R = 0; R < NT; ++R) {
            const int r = 8 * R + a;
            df t[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 ph = cur[(R * 4 + c) * 32 + lane];
                t[c] = df{ph.x, ph.y};
                if (j > 0) {
                    const float2 pv = prv[(R * 4 + c) * 32 + lane];
                    t[c] = df_add(t[c], df{-pv.x, -pv.y});
                }
                if (src && r < b) {
                    const int sh = 4 * q + c;
                    const float pv = src[((long long)j * b + r) * 16 + 2 * (sh & 7) + (sh >> 3)];
                    const float f = __fmul_rn(pv, w[c]);
                    t[c] = df_add(t[c], df{f, fmaf(pv, w[c], -f)});
                }
            }
            if (j == 0) {
                if (r < b) stg2_row(Mq, r, q, t);               // (2.1) face data
            } else {
                float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
                if (r < b) {
                    x0 = make_float4(t[0].hi, t[0].lo, t[1].hi, t[1].lo);
                    x1 = make_float4(t[2].hi, t[2].lo, t[3].hi, t[3].lo);
                }
                *reinterpret_cast<float4*>(X + r * P2ROW + 8 * q) = x0;
                *reinterpret_cast<float4*>(X + r * P2ROW + 8 * q + 4) = x1;
            }
        }
        if (j == 0) continue;
        __syncwarp();
        tl = ring_take(ring, stages, stage_elems, full, p);
        if (tl) sym2_to<NT>(tl, X, prv);                       // a_j (over phi_{j-1})
        ring_give(ring, empty, p.nstage);
        if (!tl) continue;
        // (2.2) increment and state update, Eq. (19)
        float* Dj = D + j * lb;
        float* Ujw = U + j * lb;
#pragma unroll
        for (int R = 0; R < NT; ++R) {
            const int r = 8 * R + a;
            if (r < b) {
                float4 d0, d1, u0, u1;
                ldg2_row(Dj, r, q, d0, d1);
                ldg2_row(Ujw, r, q, u0, u1);
                df dd[4], uu[4];
                unpack4(d0, d1, dd);
                unpack4(u0, u1, uu);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 av = prv[(R * 4 + c) * 32 + lane];
                    dd[c] = df_add(dd[c], df_mul(dt2, df{av.x, av.y}));
                    uu[c] = df_add(uu[c], dd[c]);
                }
                stg2_row(Dj, r, q, dd);
                stg2_row(Ujw, r, q, uu);
            }
        }
    }
    __syncwarp();
    if (nrp > 0) flush_readout2(p, g, n, rp0, nrp, acc);
}

// Readout of the final sample from the state in global memory.
template <int NT>
__device__ void unit_final_readout2(const PanelParams& p, int s, int g, int b, int k, float* acc) {
    const int rp0 = p.sub_rp_ptr[s], nrp = p.sub_rp_ptr[s + 1] - rp0;
    if (nrp == 0) return;
    const float* U = p.U + ((long long)g * p.nstate + p.state_off[s]) * 32;
    for (int j = 0; j < k; ++j) readout_level2<NT>(p, U, b, j, rp0, nrp, acc);
    flush_readout2(p, g, p.nsteps, rp0, nrp, acc);
}

// Phase B of unit (g, s) in two-float form (see unit_b): face sums of both
// sides, a_f = H_f sum (compensated), level-0 update.
__device__ void unit_b2(const PanelParams& p, int s, int g, int b, int n, const float* mail, float* scr) {
    const int lane = threadIdx.x & 31;
    const long long mrow = p.mail_off[s];
    const long long mg = (long long)g * p.nmail;
    const df dt2 = {p.dt2, p.dt2lo};
    for (int i = lane; i < b * 16; i += 32) {
        const int r = i >> 4, c = i & 15;
        const int4 e = p.frow[mrow + r];
        const float2 m0 = *reinterpret_cast<const float2*>(mail + ((mg + mrow + r) * 16 + c) * 2);
        df v = {m0.x, m0.y};
        if (e.x >= 0) {
            const float2 m1 = *reinterpret_cast<const float2*>(mail + ((mg + e.x) * 16 + c) * 2);
            const df o = {m1.x, m1.y};
            v = (e.z >> 16) ? df_add(o, v) : df_add(v, o);
        }
        *reinterpret_cast<float2*>(scr + 2 * i) = make_float2(v.hi, v.lo);
    }
    __syncwarp();
    const long long so = ((long long)g * p.nstate + p.state_off[s]) * 32;
    for (int i = lane; i < b * 16; i += 32) {
        const int r = i >> 4, c = i & 15;
        const int4 e = p.frow[mrow + r];
        const int m = e.z & 0xffff;
        const float* H = p.H + 2LL * e.y;
        const float* vv = scr + 2 * (e.w * 16 + c);
        float sa = 0.f, ea = 0.f;
        for (int cc = 0; cc < m; ++cc) {
            const float2 hv = *reinterpret_cast<const float2*>(H + 2LL * cc * m);
            const float2 xv = *reinterpret_cast<const float2*>(vv + 32 * cc);
            x2_fma(sa, ea, hv.x, hv.y, xv.x, xv.y);
        }
        float2* dp = reinterpret_cast<float2*>(p.dU + so + 2 * i);
        float2* up = reinterpret_cast<float2*>(p.U + so + 2 * i);
        const float2 d0 = *dp, u0 = *up;
        const df d = df_add(df{d0.x, d0.y}, df_mul(dt2, x2_norm(sa, ea)));
        const df un = df_add(df{u0.x, u0.y}, d);
        *dp = make_float2(d.hi, d.lo);
        *up = make_float2(un.hi, un.lo);
        if (!(fabsf(un.hi) < 1e30f)) {
            if (p.ustep) atomicMin(p.ustep, n);
            atomicCAS(p.err, 0, (int)SFM_ERR_UNSTABLE);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void unit_a2_any(int nt, const PanelParams& p, int s, int g, int b, int k, int n,
                                            float* mail, float* acc, float* slots, Ring& ring,
                                            const float* stages, int stage_elems,
                                            unsigned long long* full, unsigned long long* empty) {
    switch (nt) {
        case 1: unit_a2<1>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 2: unit_a2<2>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 3: unit_a2<3>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 4: unit_a2<4>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 5: unit_a2<5>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 6: unit_a2<6>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        case 7: unit_a2<7>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
        default: unit_a2<8>(p, s, g, b, k, n, mail, acc, slots, ring, stages, stage_elems, full, empty); break;
    }
}

__device__ __forceinline__ void final_readout2_any(int nt, const PanelParams& p, int s, int g, int b, int k,
                                                   float* acc) {
    switch (nt) {
        case 1: unit_final_readout2<1>(p, s, g, b, k, acc); break;
        case 2: unit_final_readout2<2>(p, s, g, b, k, acc); break;
        case 3: unit_final_readout2<3>(p, s, g, b, k, acc); break;
        case 4: unit_final_readout2<4>(p, s, g, b, k, acc); break;
        case 5: unit_final_readout2<5>(p, s, g, b, k, acc); break;
        case 6: unit_final_readout2<6>(p, s, g, b, k, acc); break;
        case 7: unit_final_readout2<7>(p, s, g, b, k, acc); break;
        default: unit_final_readout2<8>(p, s, g, b, k, acc); break;
    }
}

// Floats of a warp's shared-memory region in two-float mode: the product
// input X (bpad rows of P2ROW floats) and two product outputs (4 nt pairs a
// lane each, 32 bpad floats).
__host__ __device__ inline long long warp_region2_floats(int bmax) {
    const long long bpad = ((bmax + 7) / 8) * 8;
    return (bpad * P2ROW + bpad * 64 + 31) / 32 * 32;
}

// The persistent two-float panel kernel: panel_kernel's structure (tasks,
// producer ring, device-wide barrier, face phase) with the two-float units.
// at most four consumer warps and the producer; two blocks an SM (168 registers)
__global__ void __launch_bounds__(160, 2) panel2_kernel(const __grid_constant__ PanelParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ncw = p.ncw, nct = ncw * 32, nstage = p.nstage;
    const int stage_elems = (int)(tri_tiles(p.bmax) * P2TILE);
    float* stages = reinterpret_cast<float*>(smem_raw);
    const long long wreg = warp_region2_floats(p.bmax);
    float* slot_all = stages + (size_t)nstage * stage_elems;
    float* acc_all = slot_all + (size_t)ncw * wreg;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(acc_all + (size_t)ncw * p.rpmax * 32) + 15) & ~(uintptr_t)15);
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
    for (int i = threadIdx.x; i < ncw * p.rpmax * 32; i += blockDim.x) acc_all[i] = 0.f;
    __syncthreads();

    if (warp == ncw) {
        // producer: the task's blocks Gamma_0, Gamma_1, Gammahat_1, ...
        if (lane != 0) return;
        long long gcount = 0;
        int st = 0;
        unsigned ph = 0;
        bool ok = true;
        for (int n = 0; n < p.nsteps && ok; ++n) {
            for (int tk = tk0; tk < tk1 && ok; ++tk) {
                const int4 T = p.task[tk];
                const int b = T.w & 255, k = T.w >> 8;
                const long long ltile = tri_tiles(b) * P2TILE;
                const unsigned bytes = (unsigned)(ltile * sizeof(float));
                const long long base = p.coef_off[T.x];
                for (int m = 0; m < 2 * k - 1; ++m, ++gcount) {
                    if (gcount >= nstage && !mbar_wait(empty + st, ph ^ 1u, p.err, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    const long long off = base + (m == 0 ? 0 : (long long)(m + 1)) * ltile;
                    mbar_expect_tx(full + st, bytes);
                    bulk_g2s(stages + (size_t)st * stage_elems, p.coef + off, bytes, full + st);
                    if (++st == nstage) { st = 0; ph ^= 1u; }
                }
            }
        }
        for (long long h = (gcount > nstage ? gcount - nstage : 0); h < gcount; ++h)
            mbar_wait(full + (int)(h % nstage), (unsigned)((h / nstage) & 1), p.err, p.timeout_ns);
        return;
    }

    float* slots = slot_all + (size_t)warp * wreg;
    float* scr = slots;                      // phase B's face sums use the product-input slot
    float* acc = acc_all + (size_t)warp * p.rpmax * 32;   // (hi, lo) pairs
    Ring ring{0, 0u, false};
    for (int n = 0; n < p.nsteps; ++n) {
        float* mail = (n & 1) ? p.mail1 : p.mail0;
        for (int tk = tk0; tk < tk1; ++tk) {
            const int4 T = p.task[tk];
            const int s = T.x, b = T.w & 255, k = T.w >> 8;
            if (warp < T.z) {
                unit_a2_any((b + 7) >> 3, p, s, T.y + warp, b, k, n, mail, acc, slots, ring, stages,
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
            if (warp < T.z) unit_b2(p, T.x, T.y + warp, T.w & 255, n, mail, scr);
        }
    }
    for (int tk = tk0; tk < tk1; ++tk) {
        const int4 T = p.task[tk];
        const int b = T.w & 255;
        if (warp < T.z) final_readout2_any((b + 7) >> 3, p, T.x, T.y + warp, b, T.w >> 8, acc);
    }
}

size_t panel_smem_bytes(int mode, int ncw, int nstage, int bmax, int rpmax) {
    size_t floats;
    if (mode == 2)
        floats = (size_t)nstage * tri_tiles(bmax) * P2TILE + (size_t)ncw * warp_region2_floats(bmax);
    else
        floats = (size_t)nstage * tri_tiles(bmax) * PTILE + (size_t)ncw * warp_region_floats(bmax, rpmax);
    size_t bytes = sizeof(float) * (floats + (size_t)ncw * rpmax * (mode == 2 ? 32 : 16));
    bytes = (bytes + 15) & ~(size_t)15;
    return bytes + 2 * (size_t)nstage * sizeof(unsigned long long);
}

template <class F>
static int panel_max_grid_f(F kernel, int ncw, size_t smem, int* grid_out) {
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // a shape that does not fit is "no grid"; its errors are cleared
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (ncw + 1) * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (per_sm < 1) return -1;
    *grid_out = per_sm * nsm;
    return 0;
}

int panel_max_grid(int mode, int ncw, size_t smem, int* grid_out) {
    if (mode == 2) return panel_max_grid_f(panel2_kernel, ncw, smem, grid_out);
    return mode == 3 ? panel_max_grid_f(panel_kernel<3>, ncw, smem, grid_out)
                     : panel_max_grid_f(panel_kernel<1>, ncw, smem, grid_out);
}

template <class F>
static cudaError_t launch_panel_f(F kernel, int mode, const PanelParams& p, int grid, cudaStream_t st) {
    const size_t smem = panel_smem_bytes(mode, p.ncw, p.nstage, p.bmax, p.rpmax);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    PanelParams pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((void*)kernel, dim3(grid), dim3((p.ncw + 1) * 32), args, smem, st);
}

cudaError_t launch_panel(int mode, const PanelParams& p, int grid, cudaStream_t st) {
    if (mode == 2) return launch_panel_f(panel2_kernel, 2, p, grid, st);
    return mode == 3 ? launch_panel_f(panel_kernel<3>, 3, p, grid, st) : launch_panel_f(panel_kernel<1>, 1, p, grid, st);
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

// Two-float padded tiles of the symmetric blocks (SFM_FP32X2P): per
// subdomain every level's Gamma_j and Gammahat_j as the upper triangle of
// 8x8 tiles (tile order of pack_tiles_kernel), 72 (hi, lo) pairs per tile:
// row r, column c at 9r + c, column 8 and everything beyond b zero.
__global__ void pack_sym2_kernel(const double* master, const long long* master_off,
                                 const long long* tile_off, const int* sub_b, const int* sub_k, float* out) {
    const int s = blockIdx.y;
    const int b = sub_b[s], k = sub_k[s];
    const int nt = (b + 7) / 8, T = nt * (nt + 1) / 2;
    const long long total = 2LL * k * T * 72;
    const double* m = master + master_off[s];
    float* o = out + tile_off[s] / 64 * P2TILE;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int el = (int)(e % 72);
        long long rest = e / 72;
        const int tix = (int)(rest % T);
        rest /= T;
        const int which = (int)(rest & 1), j = (int)(rest >> 1);
        int I = 0, base = 0;
        while (base + (nt - I) <= tix) { base += nt - I; ++I; }
        const int J = I + (tix - base);
        const int r = el / 9, c = el % 9;
        const int row = 8 * I + r, col = 8 * J + c;
        double v = 0.0;
        if (c < 8 && row < b && col < b) v = m[((long long)which * k + j) * b * b + (long long)row * b + col];
        const float hi = (float)v;
        o[2 * e] = hi;
        o[2 * e + 1] = (float)(v - (double)hi);
    }
}

cudaError_t launch_pack_sym2(const double* master, const long long* master_off, const long long* tile_off,
                             const int* sub_b, const int* sub_k, int nsub, float* out, cudaStream_t st) {
    for (int s0 = 0; s0 < nsub; s0 += 65535) {
        const int ns = std::min(65535, nsub - s0);
        pack_sym2_kernel<<<dim3(64, ns), 256, 0, st>>>(master, master_off + s0, tile_off + s0, sub_b + s0,
                                                       sub_k + s0, out);
    }
    return cudaGetLastError();
}

// FP64 [nshots][n] <-> two-float panels [ngroups][n][16 shots][hi, lo]
// (natural shot order; padded shots zero).
__global__ void to_panel2_kernel(const double* in, float* out, int nshots, long long n, int ngroups) {
    const long long total = (long long)ngroups * n * 16;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i & 15);
        const long long ge = i >> 4;
        const int g = (int)(ge / n);
        const long long e = ge - (long long)g * n;
        const int q = 16 * g + c;
        const double v = q < nshots ? in[(long long)q * n + e] : 0.0;
        const float hi = (float)v;
        out[2 * i] = hi;
        out[2 * i + 1] = (float)(v - (double)hi);
    }
}

cudaError_t launch_to_panel2(const double* in, float* out, int nshots, long long n, cudaStream_t st) {
    const int ngroups = (nshots + 15) / 16;
    const long long total = (long long)ngroups * n * 16;
    const int grid = (int)std::min<long long>(std::max<long long>((total + 255) / 256, 1), 8192);
    to_panel2_kernel<<<grid, 256, 0, st>>>(in, out, nshots, n, ngroups);
    return cudaGetLastError();
}

__global__ void from_panel2_kernel(const float* in, double* out, int nshots, long long n) {
    const long long total = (long long)nshots * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / n);
        const long long e = i - (long long)q * n;
        const long long at = (((long long)(q >> 4)) * n + e) * 16 + (q & 15);
        out[i] = (double)in[2 * at] + (double)in[2 * at + 1];
    }
}

cudaError_t launch_from_panel2(const float* in, double* out, int nshots, long long n, cudaStream_t st) {
    const long long total = (long long)nshots * n;
    const int grid = (int)std::min<long long>(std::max<long long>((total + 255) / 256, 1), 8192);
    from_panel2_kernel<<<grid, 256, 0, st>>>(in, out, nshots, n);
    return cudaGetLastError();
}

// Traces from the two-float partial sums of mode 2 ([g][n][pair][pos]
// (hi, lo) pairs, positions as flush_readout2 writes them), summed in FP64.
__global__ void panel_traces2_kernel(const float* partial, const int* rec_ptr, const int* rec_pairs,
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
        for (int e = rec_ptr[r]; e < rec_ptr[r + 1]; ++e) {
            const long long at = (row + rec_pairs[e]) * 16 + pos;
            acc += (double)partial[2 * at] + (double)partial[2 * at + 1];
        }
        traces[i] = acc;
        if (!isfinite(acc)) atomicExch(bad, 1);
    }
}

cudaError_t launch_panel_traces2(const float* partial, const int* rec_ptr, const int* rec_pairs,
                                 int nshots, int nsteps, int nrec, int nrpairs, double* traces,
                                 int* bad, cudaStream_t st) {
    const long long total = (long long)nshots * nrec * (nsteps + 1);
    const int grid = (int)std::min<long long>(std::max<long long>((total + 255) / 256, 1), 4096);
    panel_traces2_kernel<<<grid, 256, 0, st>>>(partial, rec_ptr, rec_pairs, nshots, nsteps, nrec,
                                               nrpairs, traces, bad);
    return cudaGetLastError();
}

}  // namespace sfm
