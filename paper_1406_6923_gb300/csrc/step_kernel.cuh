// The coupled stepping kernel and its device helpers (included by step.cu);
// see step.cu for the scheme.
#pragma once

#include "sfm_internal.h"

#include <cstdint>
#include <type_traits>

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

// Block layout of the stepping kernel: p.ncw consumer warps do the
// arithmetic, one producer warp streams the coefficient blocks into shared
// memory with bulk asynchronous copies (the TMA engine) through a ring of
// p.nstage stages.  Both are chosen at launch (sfm_autotune picks them).
constexpr int NCW_MAX = 8;
constexpr int STEP_BLOCK_MAX = (NCW_MAX + 1) * 32;

__device__ __forceinline__ void cbar(int nct) {
    asm volatile("bar.sync 1, %0;" ::"r"(nct) : "memory");
}

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return (unsigned)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for a phase of an mbarrier: false (with *err set) when it did
// not complete within timeout_ns or another block reported an error.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err,
                                          unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 7) == 0) {   // the error flag and the clock every 8 polls
            if (*(volatile int*)err != 0) return false;
            if (global_ns() - t0 > timeout_ns) {
                atomicCAS(err, 0, (int)SFM_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Per-thread asynchronous global -> shared copies (4 or 8 bytes): a block
// issues all copies of a piece, then waits once, instead of paying the load
// latency once per loop trip.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bounded device-wide barrier among the consumer threads of every block, in
// two halves: grid_arrive publishes the block's writes and counts it in;
// grid_wait returns once every block has arrived, or false (with *err set)
// when that did not happen within timeout_ns or another block reported an
// error; every block then leaves the kernel.  Work that reads only data
// finished before the previous barrier may run between the two halves.
__device__ __forceinline__ void grid_arrive(unsigned int* bar, int skip_arrive, int nct) {
    cbar(nct);
    if (threadIdx.x == 0) {
        __threadfence();
        if ((int)blockIdx.x != skip_arrive) red_release_add_u32(bar, 1u);
    }
}

__device__ inline bool grid_wait(unsigned int* bar, unsigned int target, int* err,
                          unsigned long long timeout_ns, int nct) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
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
    cbar(nct);
    return s_ok != 0;
}

__device__ inline bool grid_barrier(unsigned int* bar, unsigned int target, int* err,
                             unsigned long long timeout_ns, int skip_arrive, int nct) {
    grid_arrive(bar, skip_arrive, nct);
    return grid_wait(bar, target, err, timeout_ns, nct);
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

// Receiver readout of U (buffer `Ubuf`) at sample n.  Every (shot, pair)
// item is one warp's dot product (policy arithmetic) of the pair's row with
// the subdomain's state.  Warps take items two at a time from the sample's
// counter p.rctr[n] (zero at launch), so blocks with idle time take more.
template <class P>
__device__ void readout(const StepParams<typename P::S>& p, const typename P::S* Ubuf, int n) {
    using C = typename P::C;
    const int items = p.nshots * p.nrpairs;
    if (items == 0) return;
    const int lane = threadIdx.x & 31;
    constexpr int CHUNK = 2;
    for (;;) {
        int base = 0;
        if (lane == 0) base = (int)atomicAdd(p.rctr + n, (unsigned)CHUNK);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= items) break;
        const int iend = base + CHUNK < items ? base + CHUNK : items;
        for (int it = base; it < iend; ++it) {
            const int q = it / p.nrpairs, r = it - q * p.nrpairs;
            const int4 e = p.rtab[r];
            const int kb = e.x;
            const typename P::S* row = p.rrows + e.y;
            const typename P::S* U = Ubuf + q * p.state_stride + e.z;
            C v;
            if constexpr (sizeof(typename P::S) == 4) {
                // FP32 rows and state: 16-byte loads, all of a lane's loads in
                // flight at once when k*b is a multiple of 4 and both are aligned
                if ((kb & 3) == 0 && ((reinterpret_cast<uintptr_t>(row) | reinterpret_cast<uintptr_t>(U)) & 15) == 0) {
                    const float4* r4 = reinterpret_cast<const float4*>(row);
                    const float4* u4 = reinterpret_cast<const float4*>(U);
                    float a0 = 0.f, a1 = 0.f;
    #pragma unroll 8
                    for (int t = lane; t < (kb >> 2); t += 32) {
                        const float4 x = r4[t], y = u4[t];
                        a0 = fmaf(x.x, y.x, a0);
                        a1 = fmaf(x.y, y.y, a1);
                        a0 = fmaf(x.z, y.z, a0);
                        a1 = fmaf(x.w, y.w, a1);
                    }
                    v = a0 + a1;
                } else {
                    float a0 = 0.f;
                    for (int t = lane; t < kb; t += 32) a0 = fmaf(row[t], U[t], a0);
                    v = a0;
                }
            } else {
                typename P::Acc a0 = P::acc0(), a1 = P::acc0();
                int t = lane;
    #pragma unroll 4
                for (; t + 32 < kb; t += 64) {
                    P::fma(a0, P::ld(row + t), P::ld(U + t));
                    P::fma(a1, P::ld(row + t + 32), P::ld(U + t + 32));
                }
                if (t < kb) P::fma(a0, P::ld(row + t), P::ld(U + t));
                v = P::get(P::merge(a0, a1));
            }
            for (int o = 16; o > 0; o >>= 1) v = P::add(v, P::shfl_xor(v, o));
            if (lane == 0) P::st(p.partial + ((long long)q * (p.nsteps + 1) + n) * p.nrpairs + r, v);
        }
    }
}

// One tile row of y = M x for a symmetric block M held in shared memory as
// its upper triangle of 8x8 tiles (tile (I,J), J >= I, at index
// I*nt - I(I-1)/2 + (J-I), row-major inside the tile).  Lane (r, q) sums
// row 8I+r over columns 8J+2q, 8J+2q+1 of every tile column J; a tile below
// the diagonal is read transposed from its stored mirror.
template <class P>
__device__ __forceinline__ void tile_row(const typename P::S* tiles, int nt, int I,
                                         const typename P::C* x, typename P::C* y) {
    using C = typename P::C;
    const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
    // two independent accumulators (even and odd tile columns) for ILP
    typename P::Acc a0 = P::acc0(), a1 = P::acc0();
    auto load = [&](int J, C& e0, C& e1) {
        if (J >= I) {
            P::ld2p(tiles + (I * nt - I * (I - 1) / 2 + (J - I)) * 64 + r * 8 + 2 * q, e0, e1);
        } else {
            const typename P::S* t = tiles + (J * nt - J * (J - 1) / 2 + (I - J)) * 64;
            e0 = P::ld(t + (2 * q) * 8 + r);
            e1 = P::ld(t + (2 * q + 1) * 8 + r);
        }
    };
    int J = 0;
    for (; J + 1 < nt; J += 2) {
        C e0, e1, f0, f1;
        load(J, e0, e1);
        load(J + 1, f0, f1);
        P::fma(a0, e0, x[8 * J + 2 * q]);
        P::fma(a1, f0, x[8 * J + 8 + 2 * q]);
        P::fma(a0, e1, x[8 * J + 2 * q + 1]);
        P::fma(a1, f1, x[8 * J + 8 + 2 * q + 1]);
    }
    if (J < nt) {
        C e0, e1;
        load(J, e0, e1);
        P::fma(a0, e0, x[8 * J + 2 * q]);
        P::fma(a0, e1, x[8 * J + 2 * q + 1]);
    }
    C v = P::get(P::merge(a0, a1));
    v = P::add(v, P::shfl_xor(v, 1));
    v = P::add(v, P::shfl_xor(v, 2));
    if (q == 0) y[8 * I + r] = v;
}

// y = L (L^T x) for one S-fraction block held as its lower Cholesky factor
// L in shared memory: lower-triangular 8x8 tiles (tile (I,J), J <= I, at
// index I(I+1)/2 + J, row-major inside the tile, zero above the diagonal
// and beyond b).  One warp does the whole block.  Lane (r, q) reads the two
// consecutive elements (r, 2q), (r, 2q+1) of every tile (one conflict-free
// 8-byte load per tile per pass):
//   z = L^T x: lane sums x_{8I+r} L_IJ[r][2q..2q+1] over I >= J, then an
//              xor butterfly over r leaves z_{8J+2q}, z_{8J+2q+1} in every
//              lane of that q, which is what the second pass reads;
//   y = L z:   lane sums L_IJ[r][2q..2q+1] . z_J[2q..2q+1] over J <= I, then
//              a butterfly over q gives y_{8I+r}.
// The summation order is fixed by (nt, lane), never by the block shape.
// xf(row) gives x at a row index 8I+r (read by the lanes of that r), ef(row,
// y) receives the result in the four lanes q = 0 of each row group.  Blocks
// up to 64 wide: the loops run to 8 tiles with uniform guards, one instance
// for every width, which keeps the arrays in registers.
template <class XF, class EF>
__device__ __forceinline__ void factor_apply(int nt, const float* tiles, XF xf, EF ef) {
    constexpr int NTMAX = 8;
    const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
    const float* t0 = tiles + r * 8 + 2 * q;
    float xr[NTMAX], z0[NTMAX], z1[NTMAX];
#pragma unroll
    for (int I = 0; I < NTMAX; ++I) xr[I] = (I < nt) ? xf(8 * I + r) : 0.f;
#pragma unroll
    for (int J = 0; J < NTMAX; ++J) {
        float a0 = 0.f, a1 = 0.f;
        if (J < nt) {
#pragma unroll
            for (int I = J; I < NTMAX; ++I) {
                if (I < nt) {
                    const float2 l =
                        *reinterpret_cast<const float2*>(t0 + (I * (I + 1) / 2 + J) * 64);
                    a0 = fmaf(l.x, xr[I], a0);
                    a1 = fmaf(l.y, xr[I], a1);
                }
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            }
        }
        z0[J] = a0;
        z1[J] = a1;
    }
#pragma unroll
    for (int I = 0; I < NTMAX; ++I) {
        if (I < nt) {
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int J = 0; J <= I; ++J) {
                const float2 l = *reinterpret_cast<const float2*>(t0 + (I * (I + 1) / 2 + J) * 64);
                a0 = fmaf(l.x, z0[J], a0);
                a1 = fmaf(l.y, z1[J], a1);
            }
            float v = a0 + a1;
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (q == 0) ef(8 * I + r, v);
        }
    }
}

// The same product for a fixed tile count: no guards, so the compiler can
// interleave the independent reductions of the tile columns and rows.
template <int NT, class XF, class EF>
__device__ __forceinline__ void factor_apply_nt(const float* tiles, XF xf, EF ef) {
    const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
    const float* t0 = tiles + r * 8 + 2 * q;
    float xr[NT], z0[NT], z1[NT];
#pragma unroll
    for (int I = 0; I < NT; ++I) xr[I] = xf(8 * I + r);
#pragma unroll
    for (int J = 0; J < NT; ++J) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int I = J; I < NT; ++I) {
            const float2 l = *reinterpret_cast<const float2*>(t0 + (I * (I + 1) / 2 + J) * 64);
            a0 = fmaf(l.x, xr[I], a0);
            a1 = fmaf(l.y, xr[I], a1);
        }
        z0[J] = a0;
        z1[J] = a1;
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
#pragma unroll
        for (int J = 0; J < NT; ++J) {
            z0[J] += __shfl_xor_sync(0xffffffffu, z0[J], o);
            z1[J] += __shfl_xor_sync(0xffffffffu, z1[J], o);
        }
    }
    float v[NT];
#pragma unroll
    for (int I = 0; I < NT; ++I) {
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int J = 0; J <= I; ++J) {
            const float2 l = *reinterpret_cast<const float2*>(t0 + (I * (I + 1) / 2 + J) * 64);
            a0 = fmaf(l.x, z0[J], a0);
            a1 = fmaf(l.y, z1[J], a1);
        }
        v[I] = a0 + a1;
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
#pragma unroll
        for (int I = 0; I < NT; ++I) v[I] += __shfl_xor_sync(0xffffffffu, v[I], o);
    }
    if (q == 0) {
#pragma unroll
        for (int I = 0; I < NT; ++I) ef(8 * I + r, v[I]);
    }
}

template <class XF, class EF>
__device__ __forceinline__ void factor_apply_any(int nt, const float* tiles, XF xf, EF ef) {
    if (nt == 6) factor_apply_nt<6>(tiles, xf, ef);
    else factor_apply(nt, tiles, xf, ef);
}

// The product of factor_apply for two-float vectors (PolF32Fx2): the same
// lanes, tile loads and summation order, with every sum compensated
// (PolF32Fx2::fma1 per product, two-float butterflies), so that the FP32
// factor elements are the only rounded operands.  NT is the largest tile
// count; nt <= NT the block's.
template <int NT, class XF, class EF>
__device__ __forceinline__ void factor_apply2_nt(int nt, const float* tiles, XF xf, EF ef) {
    using P = PolF32Fx2;
    const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
    const float* t0 = tiles + r * 8 + 2 * q;
    df xr[NT], z0[NT], z1[NT];
#pragma unroll
    for (int I = 0; I < NT; ++I) xr[I] = (I < nt) ? xf(8 * I + r) : df{0.f, 0.f};
#pragma unroll
    for (int J = 0; J < NT; ++J) {
        P::Acc a0 = P::acc0(), a1 = P::acc0();
        if (J < nt) {
#pragma unroll
            for (int I = J; I < NT; ++I) {
                if (I < nt) {
                    const float2 l =
                        *reinterpret_cast<const float2*>(t0 + (I * (I + 1) / 2 + J) * 64);
                    P::fma1(a0, l.x, xr[I]);
                    P::fma1(a1, l.y, xr[I]);
                }
            }
            // the two-sum is exact, so both lanes of each exchange get the
            // same merged value and the whole column group agrees
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                a0 = P::merge(a0, P::shfl_xor_acc(a0, o));
                a1 = P::merge(a1, P::shfl_xor_acc(a1, o));
            }
        }
        z0[J] = P::get(a0);
        z1[J] = P::get(a1);
    }
#pragma unroll
    for (int I = 0; I < NT; ++I) {
        if (I < nt) {
            P::Acc a0 = P::acc0(), a1 = P::acc0();
#pragma unroll
            for (int J = 0; J <= I; ++J) {
                const float2 l = *reinterpret_cast<const float2*>(t0 + (I * (I + 1) / 2 + J) * 64);
                P::fma1(a0, l.x, z0[J]);
                P::fma1(a1, l.y, z1[J]);
            }
            P::Acc a = P::merge(a0, a1);
            a = P::merge(a, P::shfl_xor_acc(a, 1));
            a = P::merge(a, P::shfl_xor_acc(a, 2));
            if (q == 0) ef(8 * I + r, P::get(a));
        }
    }
}

template <class XF, class EF>
__device__ __forceinline__ void factor_apply2_any(int nt, const float* tiles, XF xf, EF ef) {
    if (nt == 6) factor_apply2_nt<6>(6, tiles, xf, ef);
    else factor_apply2_nt<8>(nt, tiles, xf, ef);
}

// Coefficient tiles the producer streams: the packed blocks, or the factor
// tiles for the factored policies.
template <class P>
__device__ __forceinline__ const typename P::K* coef_base(const StepParams<typename P::S>& p) {
    if constexpr (P::factored) return p.fcoef;
    else return p.coef;
}

// Work of one block per time step: a list of pieces (unit, j0, j1), each a
// contiguous range of levels of one (shot, subdomain) unit.  A piece streams
// Gamma_j for j in [max(j0-1, 0), j1) (the extra level j0-1 gives phi_{j0-1},
// needed by psi_{j0}) and then Gammahat_j for j in [max(j0, 1), j1); it
// updates levels [max(j0, 1), j1) and, when j0 = 0, owns the unit's faces.
__device__ __forceinline__ int piece_blocks(int j0, int j1) {
    return (j1 - (j0 > 0 ? j0 - 1 : 0)) + (j1 - (j0 > 1 ? j0 : 1));
}

template <class P>
__global__ void __launch_bounds__(step_max_threads<P>(), step_min_blocks<P>()) step_kernel(StepParams<typename P::S> p) {
    using S = typename P::S;
    using C = typename P::C;
    using K = typename P::K;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ncw = p.ncw, nct = ncw * 32, nstage = p.nstage;
    const int bpm = ((p.bmax + 7) / 8) * 8;
    const int stage_elems = (int)(sym_tiles(p.bmax) * 64);
    K* stages = reinterpret_cast<K*>(smem_raw);
    // Per-piece staging: the factored path double-buffers the state,
    // increment and source rows (set 1 at +SU / +SD) so the next piece loads
    // while the current one computes.
    constexpr int NSET = P::factored ? 2 : 1;
    const int SU = (p.kmax + 1) * bpm, SD = p.kmax * bpm;
    C* sU = reinterpret_cast<C*>(stages + (size_t)nstage * stage_elems);   // NSET x (kmax+1)*bpm
    C* sD = sU + NSET * SU;                              // NSET x kmax*bpm: Delta/psi or increments
    C* sPhi = sD + NSET * SD;                            // kmax*bpm: phi, then a; face sums
    C* sSrc = sPhi + SD;                                 // NSET x kmax*bpm: source rows (factored)
    C* sEnd = P::factored ? sSrc + NSET * SD : sSrc;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(sEnd) + 15) & ~(uintptr_t)15);
    unsigned long long* empty = full + nstage;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pc0 = p.piece_ptr[blockIdx.x], pc1 = p.piece_ptr[blockIdx.x + 1];
    // the block's first piece records, cached in shared memory
    constexpr int REC_CACHE = 8;
    __shared__ int4 s_rec[2 * REC_CACHE];
    for (int t = threadIdx.x; t < 2 * min(pc1 - pc0, REC_CACHE); t += blockDim.x)
        s_rec[t] = p.prec[2 * pc0 + t];
    auto prec = [&](int pc, int half) -> int4 {
        return (pc - pc0 < REC_CACHE) ? s_rec[2 * (pc - pc0) + half] : p.prec[2 * pc + half];
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < nstage; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, P::factored ? 1 : ncw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == ncw) {
        // ------------------------------ producer ------------------------------
        if (lane != 0) return;
        long long g = 0;
        int st = 0;            // stage of block g = g % nstage
        unsigned ph = 0;       // parity of that stage's current use = (g / nstage) & 1
        bool ok = true;
        for (int n = 0; n < p.nsteps && ok; ++n) {
            for (int pc = pc0; pc < pc1 && ok; ++pc) {
                const int4 r0 = prec(pc, 0), r1 = prec(pc, 1);
                const int s = r0.y, j0 = r0.z, j1 = r0.w;
                const int b = r1.x & 255;
                const int nt = (b + 7) >> 3;
                const long long ltile = 2LL * (nt * (nt + 1) / 2) * 64;
                const unsigned bytes = (unsigned)((ltile / 2) * sizeof(K));
                const long long T0 = p.coef_off[s];
                const int jl = j0 > 0 ? j0 - 1 : 0, ja = j0 > 1 ? j0 : 1;
                const int nblk = piece_blocks(j0, j1);
                for (int m = 0; m < nblk; ++m, ++g) {
                    // the stage's previous use (block g - nstage) must be released
                    if (g >= nstage && !mbar_wait(empty + st, ph ^ 1u, p.err, p.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    const long long off = (m < j1 - jl) ? T0 + (long long)(jl + m) * ltile
                                                        : T0 + (long long)(ja + m - (j1 - jl)) * ltile + ltile / 2;
                    mbar_expect_tx(full + st, bytes);
                    bulk_g2s(stages + (size_t)st * stage_elems, coef_base<P>(p) + off, bytes, full + st);
                    if (++st == nstage) { st = 0; ph ^= 1u; }
                }
            }
        }
        // never leave with copies in flight: wait for every issued stage
        for (long long h = (g > nstage ? g - nstage : 0); h < g; ++h)
            mbar_wait(full + (int)(h % nstage), (unsigned)((h / nstage) & 1), p.err, p.timeout_ns);
        return;
    }

    // ------------------------------- consumers --------------------------------
    const C dt2 = P::from_d(p.dt2);
    // Running position in the stream of blocks (same order as the producer):
    // stage cst = g % nstage, parity cph = (g / nstage) & 1 of its use, and
    // for factored blocks the owner warp own = g % ncw (ncw divides nstage,
    // so every stage always has the same owner, which waits for each of its
    // phases in order: a warp never waits on a stage more than one phase
    // ahead of the producer).  A failed bounded wait marks the warp dead: it
    // skips its remaining waits and arithmetic but keeps taking part in the
    // block's named barriers, and the next device-wide barrier, which sees
    // the error flag, sends every warp out together.
    int cst = 0, own = 0;
    unsigned cph = 0;
    bool dead = false;
    // factored path: issue the copies of piece pcx into staging set `set`
    // (one cp.async group per call; zero padding written directly).  With
    // skip0 the level-0 rows of U are left to the caller (phase B computes
    // them in this block and writes them into the set itself).
    constexpr int EPV = (int)(16 / sizeof(S));   // state elements per 16-byte copy
    auto stage = [&](int pcx, int set, const S* Ubuf, bool skip0) {
        const int4 a0 = prec(pcx, 0), a1 = prec(pcx, 1);
        const int xj0 = a0.z, xj1 = a0.w, xb = a1.x & 255, xk = a1.x >> 8;
        const int xbp = ((xb + 7) >> 3) * 8;
        const int xjl = xj0 > 0 ? xj0 - 1 : 0, xja = xj0 > 1 ? xj0 : 1, xnl = xj1 - xjl;
        const long long xso = a0.x * p.state_stride + a1.y, xsof = a1.z;
        C* xU = sU + set * SU;
        C* xD = sD + set * SD;
        C* xS = sSrc + set * SD;
        if (p.stage_v4) {
            // every width a multiple of EPV: 16-byte copies, zero padding
            // from b to the tile width and for level k (if reached)
            for (int lj = warp; lj <= xnl; lj += ncw) {
                const int j = xjl + lj;
                for (int i = EPV * lane; i < xbp; i += 32 * EPV) {
                    if (j < xk && i < xb) {
                        if (!(skip0 && j == 0)) cp_async<16>(xU + lj * xbp + i, Ubuf + xso + j * xb + i);
                    } else {
                        *reinterpret_cast<float4*>(xU + lj * xbp + i) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            for (int lj = xja - xjl + warp; lj < xnl; lj += ncw) {
                const int j = xjl + lj;
                for (int i = EPV * lane; i < xb; i += 32 * EPV)
                    cp_async<16>(xD + lj * xbp + i, p.dU + xso + j * xb + i);
            }
            if (xsof >= 0) {
                for (int lj = warp; lj < xnl; lj += ncw) {
                    const int j = xjl + lj;
                    for (int i = EPV * lane; i < xb; i += 32 * EPV)
                        cp_async<16>(xS + lj * xbp + i, p.src + xsof + j * xb + i);
                }
            }
            cp_async_commit();
            return;
        }
        for (int lj = warp; lj <= xnl; lj += ncw) {
            const int j = xjl + lj;
            for (int i = lane; i < xbp; i += 32) {
                if (j < xk && i < xb) {
                    if (!(skip0 && j == 0)) cp_async<sizeof(S)>(xU + lj * xbp + i, Ubuf + xso + j * xb + i);
                } else {
                    xU[lj * xbp + i] = P::zero();
                }
            }
        }
        for (int lj = xja - xjl + warp; lj < xnl; lj += ncw) {
            const int j = xjl + lj;
            for (int i = lane; i < xb; i += 32)
                cp_async<sizeof(S)>(xD + lj * xbp + i, p.dU + xso + j * xb + i);
        }
        if (xsof >= 0) {
            for (int lj = warp; lj < xnl; lj += ncw) {
                const int j = xjl + lj;
                for (int i = lane; i < xb; i += 32)
                    cp_async<sizeof(S)>(xS + lj * xbp + i, p.src + xsof + j * xb + i);
            }
        }
        cp_async_commit();
    };
    bool pre = false;   // the first piece of this step was staged during the last step's phase B
    for (int n = 0; n < p.nsteps; ++n) {
        const S* Ucur = p.U[n & 3];
        S* Unxt = p.U[(n + 1) & 3];
        S* mail = (n & 1) ? p.mail1 : p.mail0;

        // ---------------- phase A ----------------
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 r0 = prec(pc, 0), r1 = prec(pc, 1);
            const int q = r0.x, j0 = r0.z, j1 = r0.w;
            const int b = r1.x & 255, k = r1.x >> 8;
            const int nt = (b + 7) >> 3, bp = nt * 8;
            const int jl = j0 > 0 ? j0 - 1 : 0, ja = j0 > 1 ? j0 : 1, nl = j1 - jl;
            const long long so = q * p.state_stride + r1.y;
            const S* Uc = Ucur + so;
            S* Un = Unxt + so;
            S* dU = p.dU + so;
            const long long sof = r1.z;
            const long long mo = q * p.mail_stride + r1.w;
            const C w = P::ld(p.wavelet + (long long)q * p.nsteps + n);
            static_assert(sizeof(C) == sizeof(S), "state copies are byte copies");
            if constexpr (P::factored) {
                const int set = (pc - pc0) & 1;
                cbar(nct);
                if (pc == pc0 && !pre) stage(pc, set, Ucur, false);
                if (pc + 1 < pc1) stage(pc + 1, set ^ 1, Ucur, false);
                if (pc + 1 < pc1) {
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                cbar(nct);
                C* const sUs = sU + set * SU;
                C* const sDs = sD + set * SD;
                C* const sSs = sSrc + set * SD;
                // One warp per streamed block (the owner of its stage).  The
                // Gamma_j owner forms Delta_j = U_{j+1} - U_j as it loads it
                // and leaves phi_j = L L^T Delta_j in sPhi; after the barrier
                // the Gammahat_j owner forms psi_j = phi_j - phi_{j-1} + p_j f
                // the same way and applies the increment update (Eq. 19) to
                // its rows directly from the matvec.
                const bool has_src = sof >= 0;
                for (int half = 0; half < 2; ++half) {
                    const int lo = half ? ja : jl;
                    for (int j = lo; j < j1; ++j) {
                        const int st = cst, owner = own;
                        const unsigned ph = cph;
                        if (++cst == nstage) { cst = 0; cph ^= 1u; }
                        if (++own == ncw) own = 0;
                        if (owner != warp) continue;
                        if (!dead && !mbar_wait(full + st, ph, p.err, p.timeout_ns)) dead = true;
                        if (dead) continue;
                        const float* tl = reinterpret_cast<const float*>(stages) + (size_t)st * stage_elems;
                        if constexpr (sizeof(C) == sizeof(float)) {
                            const float wf = w;
                            const float* fU = reinterpret_cast<const float*>(sUs) + (j - jl) * bp;
                            float* fP = reinterpret_cast<float*>(sPhi) + (j - jl) * bp;
                            if (half == 0) {
                                factor_apply_any(nt, tl,
                                             [&](int row) { return fU[bp + row] - fU[row]; },
                                             [&](int row, float v) { fP[row] = v; });
                            } else {
                                const float* sj = reinterpret_cast<const float*>(sSs) + (j - jl) * bp;
                                const float* fD = reinterpret_cast<const float*>(sDs) + (j - jl) * bp;
                                float* dUj = reinterpret_cast<float*>(dU) + j * b;
                                float* Unj = reinterpret_cast<float*>(Un) + j * b;
                                const float d2 = (float)dt2;
                                factor_apply_any(nt, tl,
                                             [&](int row) {
                                                 float v = fP[row] - fP[row - bp];
                                                 if (has_src && row < b) v += sj[row] * wf;
                                                 return v;
                                             },
                                             [&](int row, float v) {
                                                 if (row < b) {
                                                     const float d = fD[row] + d2 * v;
                                                     dUj[row] = d;
                                                     Unj[row] = fU[row] + d;
                                                 }
                                             });
                            }
                        } else {
                            // two-float state, FP32 factor tiles (PolF32Fx2)
                            const C* fU = sUs + (j - jl) * bp;
                            C* fP = sPhi + (j - jl) * bp;
                            if (half == 0) {
                                factor_apply2_any(nt, tl,
                                                  [&](int row) { return P::sub(fU[bp + row], fU[row]); },
                                                  [&](int row, C v) { fP[row] = v; });
                            } else {
                                const C* sj = sSs + (j - jl) * bp;
                                const C* fD = sDs + (j - jl) * bp;
                                S* dUj = dU + j * b;
                                S* Unj = Un + j * b;
                                factor_apply2_any(nt, tl,
                                                  [&](int row) {
                                                      C v = P::sub(fP[row], fP[row - bp]);
                                                      if (has_src && row < b) v = P::add(v, P::mul(sj[row], w));
                                                      return v;
                                                  },
                                                  [&](int row, C v) {
                                                      if (row < b) {
                                                          const C d = P::add(fD[row], P::mul(dt2, v));
                                                          P::st(dUj + row, d);
                                                          P::st(Unj + row, P::add(fU[row], d));
                                                      }
                                                  });
                            }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(empty + st);
                    }
                    if (half == 0) {
                        cbar(nct);
                        // (2.1) publish face data [phi_1 + p_1 f]
                        if (j0 == 0) {
                            S* my_mail = mail + mo;
                            for (int i = threadIdx.x; i < b; i += nct)
                                P::st(my_mail + i, has_src ? P::add(sPhi[i], P::mul(sSs[i], w)) : sPhi[i]);
                        }
                    }
                }
            } else {
            cbar(nct);
            // padded copies of levels jl..j1 (local index = level - jl), one
            // level per warp, lanes along the level
            for (int lj = warp; lj <= nl; lj += ncw) {
                const int j = jl + lj;
                for (int i = lane; i < bp; i += 32) {
                    if (j < k && i < b) cp_async<sizeof(S)>(sU + lj * bp + i, Uc + j * b + i);
                    else sU[lj * bp + i] = P::zero();
                }
            }
            cp_async_wait_all();
            cbar(nct);
            for (int t = threadIdx.x; t < nl * bp; t += nct) sD[t] = P::sub(sU[t + bp], sU[t]);
            cbar(nct);
            // phi_j = Gamma_j Delta_j for levels jl..j1-1, then after psi,
            // a_j = Gammahat_j psi_j for levels ja..j1-1.  Tile rows of the
            // streamed blocks go to the warps round robin; every warp waits
            // for each block and releases it, so releases arrive in order.
            int task = 0;
            for (int half = 0; half < 2; ++half) {
                const int lo = half ? ja : jl;
                for (int j = lo; j < j1; ++j) {
                    const int st = cst;
                    const unsigned ph = cph;
                    if (++cst == nstage) { cst = 0; cph ^= 1u; }
                    const int lj = j - jl;
                    const int first = (warp - task % ncw + ncw) % ncw;
                    task += nt;
                    if (!dead && !mbar_wait(full + st, ph, p.err, p.timeout_ns)) dead = true;
                    if (dead) continue;
                    for (int I = first; I < nt; I += ncw)
                        tile_row<P>(stages + (size_t)st * stage_elems, nt, I, sD + lj * bp,
                                    sPhi + lj * bp);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty + st);
                }
                cbar(nct);
                if (half == 0) {
                    // (2.1) publish face data; psi_j for the updated levels
                    if (j0 == 0) {
                        S* my_mail = mail + mo;
                        for (int i = threadIdx.x; i < b; i += nct) {
                            const C srcv = (sof >= 0) ? P::mul(P::ld(p.src + sof + i), w) : P::zero();
                            P::st(my_mail + i, P::add(sPhi[i], srcv));
                        }
                    }
                    for (int lj = ja - jl + warp; lj < nl; lj += ncw) {
                        const int j = jl + lj;
                        for (int i = lane; i < b; i += 32) {
                            const C srcv = (sof >= 0) ? P::mul(P::ld(p.src + sof + j * b + i), w) : P::zero();
                            sD[lj * bp + i] = P::add(P::sub(sPhi[lj * bp + i], sPhi[(lj - 1) * bp + i]), srcv);
                        }
                    }
                    cbar(nct);
                }
            }
            // (2.2) interior update of levels ja..j1-1, Eq. (19)
            for (int lj = ja - jl + warp; lj < nl; lj += ncw) {
                const int j = jl + lj;
                for (int i = lane; i < b; i += 32) {
                    if (p.Kx) P::st(p.Kx + so + j * b + i, sD[lj * bp + i]);
                    const C d = P::add(P::ld(dU + j * b + i), P::mul(dt2, sPhi[lj * bp + i]));
                    P::st(dU + j * b + i, d);
                    P::st(Un + j * b + i, P::add(sU[lj * bp + i], d));
                }
            }
            }
        }

        // Arrive, then read out U^{n-1} (buffer (n-1) & 3, complete before
        // the previous barrier and rewritten only by phase A of step n+2,
        // after the next barrier, which needs this block) while the slower
        // blocks finish phase A, then wait.
        grid_arrive(p.bar, p.skip_arrive, nct);
        if (n > 0) readout<P>(p, p.U[(n - 1) & 3], n - 1);
        if (!grid_wait(p.bar, (unsigned)(n + 1) * gridDim.x, p.err, p.timeout_ns, nct))
            return;

        // Factored path: stage the first piece of step n+1 now, while phase
        // B runs.  Every level of U^{n+1} it reads other than level 0 was
        // written in phase A, before the barrier (a unit is never cut at
        // level 1, so only a level-0 piece reads level 0, and its face
        // update is done by this block below, which also writes those rows
        // into the staging set).
        pre = false;
        if constexpr (P::factored) {
            if (n + 1 < p.nsteps && pc0 < pc1) {
                stage(pc0, 0, Unxt, prec(pc0, 0).z == 0);
                pre = true;
            }
        }

        // ---------------- phase B: faces, Eq. (18) ----------------
        // scratch for the face rows' increments and state (a staging set the
        // next piece copies into only after the next phase A barrier)
        C* const sB = sU + (NSET - 1) * SU;
        for (int pc = pc0; pc < pc1; ++pc) {
            const int4 r0 = prec(pc, 0);
            if (r0.z != 0) continue;                     // faces belong to the level-0 piece
            const int4 r1 = prec(pc, 1);
            const int q = r0.x, b = r1.x & 255;
            const long long so = q * p.state_stride + r1.y;
            const S* mailq = mail + q * p.mail_stride;
            const int4* fr = p.frow + r1.w;
            const bool to_stage = pre && pc == pc0;
            cbar(nct);
            // sum of both sides' face data, lower subdomain index first; the
            // face rows' increment and state are loaded in the same pass
            for (int t = threadIdx.x; t < b; t += nct) {
                const int4 e = fr[t];
                C v = P::ld(mailq + r1.w + t);
                sB[t] = P::ld(p.dU + so + t);
                sB[bpm + t] = P::ld(Ucur + so + t);
                if (e.x >= 0) {
                    const C o = P::ld(mailq + e.x);
                    v = (e.z >> 16) ? P::add(o, v) : P::add(v, o);
                }
                sPhi[t] = v;
                if (p.Kx) P::st(p.Kx + so + t, v);
            }
            cbar(nct);
            for (int t = threadIdx.x; t < b; t += nct) {
                const int4 e = fr[t];
                const int m = e.z & 0xffff;
                const S* H = p.H + e.y;                  // row i of the symmetric H_f
                const C* v = sPhi + e.w;
                typename P::Acc acc = P::acc0();
                for (int c = 0; c < m; ++c) P::fma(acc, P::ld(H + c * m), v[c]);
                const C d = P::add(sB[t], P::mul(dt2, P::get(acc)));
                P::st(p.dU + so + t, d);
                const C un = P::add(sB[bpm + t], d);
                P::st(Unxt + so + t, un);
                if (to_stage) sU[t] = un;                // level 0 of staging set 0
                if (!P::sane(un)) {
                    // unstable (time step above the CFL limit): every block
                    // leaves at the next device-wide barrier
                    if (p.ustep) atomicMin(p.ustep, n);
                    atomicCAS(p.err, 0, (int)SFM_ERR_UNSTABLE);
                }
            }
        }
    }
    // the last two samples, after every face update of the last step
    grid_arrive(p.bar, p.skip_arrive, nct);
    readout<P>(p, p.U[(p.nsteps - 1) & 3], p.nsteps - 1);
    if (!grid_wait(p.bar, (unsigned)(p.nsteps + 1) * gridDim.x, p.err, p.timeout_ns, nct))
        return;
    readout<P>(p, p.U[p.nsteps & 3], p.nsteps);
}

template <class P>
size_t step_smem_bytes(int kmax, int bmax, int nstage) {
    const size_t bp = (size_t)((bmax + 7) / 8) * 8;
    size_t bytes = (size_t)nstage * sym_tiles(bmax) * 64 * sizeof(typename P::K);
    const size_t nset = P::factored ? 2 : 1;
    bytes += sizeof(typename P::C) *
             (nset * (size_t)(kmax + 1) * bp + (nset + 1 + (P::factored ? nset : 0)) * (size_t)kmax * bp);
    bytes = (bytes + 15) & ~(size_t)15;
    return bytes + 2 * nstage * sizeof(unsigned long long);
}

template <class P>
int step_max_grid(int ncw, size_t smem, int* grid_out) {
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // a shape whose shared memory does not fit is "no grid"; the failed
    // calls' errors are cleared so that no later launch check reports them
    if (cudaFuncSetAttribute(step_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<P>, (ncw + 1) * 32, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (per_sm < 1) return -1;
    *grid_out = per_sm * nsm;
    return 0;
}

template <class P>
cudaError_t launch_step(const StepParams<typename P::S>& p, int grid, cudaStream_t st) {
    const size_t smem = step_smem_bytes<P>(p.kmax, p.bmax, p.nstage);
    cudaError_t e = cudaFuncSetAttribute(step_kernel<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    StepParams<typename P::S> pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((void*)step_kernel<P>, dim3(grid), dim3((p.ncw + 1) * 32),
                                       args, smem, st);
}

}  // namespace sfm
