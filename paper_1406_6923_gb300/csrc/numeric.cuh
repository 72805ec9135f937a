// Number policies of the stepping kernels.
//
//   PolF64   : FP64 storage and arithmetic.
//   PolF32   : FP32 storage and arithmetic.
//   PolF32F  : FP32 storage and arithmetic with every S-fraction block held
//              as its Cholesky factor (Gamma = L L^T), applied as L (L^T x):
//              the factored form stays positive semi-definite whatever the
//              rounding of L, where FP32-rounded deep-ROM blocks (condition
//              numbers up to ~1e14) turn indefinite and the leapfrog diverges.
//   PolF32Fx2: FP32 Cholesky factors as in PolF32F (the same coefficient
//              bytes), with the state, the vectors of the product and its
//              sums in two-float form (below): the factors' rounding is the
//              only FP32 rounding left.
//   PolF32x2 : "two-float" numbers x = hi + lo (two FP32 words, ~48-bit
//              significand) with FP32 arithmetic made exact by error-free
//              transformations: Knuth's two-sum, the FMA two-product
//              (err = fma(a, b, -a*b)), and a compensated dot product in the
//              manner of Ogita, Rump and Oishi's Dot2 for the block
//              matrix-vector products.  GB300's FP64 rate is a small fraction
//              of its FP32 rate, so this is the fast way to step ROMs whose
//              S-fraction coefficients are too ill-conditioned for FP32.
#pragma once

#include <cuda_runtime.h>

namespace sfm {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // needs |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}

struct PolF64 {
    static constexpr bool factored = false;
    using S = double;   // storage
    using C = double;   // value in registers / shared memory
    using K = double;   // coefficient tile element
    static constexpr int kind = 0;
    __device__ static C ld(const S* p) { return *p; }
    // two consecutive elements in one 16-byte load (p 16-byte aligned)
    __device__ static void ld2(const S* p, C& a, C& b) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        a = v.x;
        b = v.y;
    }
    __device__ static C ldg(const S* p) { return __ldg(p); }
    __device__ static void ld2p(const S* p, C& a, C& b) { const double2 v = *reinterpret_cast<const double2*>(p); a = v.x; b = v.y; }
    __device__ static void st(S* p, C v) { *p = v; }
    __device__ static C add(C a, C b) { return a + b; }
    __device__ static C sub(C a, C b) { return a - b; }
    __device__ static C mul(C a, C b) { return a * b; }
    __device__ static C zero() { return 0.0; }
    __device__ static C from_d(double x) { return x; }
    __host__ __device__ static double to_d(S x) { return x; }
    // instability sentinel: false for a non-finite or runaway value
    __device__ static bool sane(C v) { return fabs(v) < 1e30; }
    __device__ static C shfl_xor(C v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    struct Acc {
        double s;
    };
    __device__ static Acc acc0() { return {0.0}; }
    __device__ static void fma(Acc& a, C x, C y) { a.s = ::fma(x, y, a.s); }
    __device__ static Acc merge(const Acc& a, const Acc& b) { return {a.s + b.s}; }
    __device__ static C get(const Acc& a) { return a.s; }
};

struct PolF32 {
    static constexpr bool factored = false;
    using S = float;
    using C = float;
    using K = float;
    static constexpr int kind = 1;
    __device__ static C ld(const S* p) { return *p; }
    __device__ static void ld2(const S* p, C& a, C& b) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        a = v.x;
        b = v.y;
    }
    __device__ static C ldg(const S* p) { return __ldg(p); }
    __device__ static void ld2p(const S* p, C& a, C& b) { const float2 v = *reinterpret_cast<const float2*>(p); a = v.x; b = v.y; }
    __device__ static void st(S* p, C v) { *p = v; }
    __device__ static C add(C a, C b) { return a + b; }
    __device__ static C sub(C a, C b) { return a - b; }
    __device__ static C mul(C a, C b) { return a * b; }
    __device__ static C zero() { return 0.f; }
    __device__ static C from_d(double x) { return (float)x; }
    __host__ __device__ static double to_d(S x) { return x; }
    __device__ static bool sane(C v) { return fabsf(v) < 1e30f; }
    __device__ static C shfl_xor(C v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    struct Acc {
        float s;
    };
    __device__ static Acc acc0() { return {0.f}; }
    __device__ static void fma(Acc& a, C x, C y) { a.s = fmaf(x, y, a.s); }
    __device__ static Acc merge(const Acc& a, const Acc& b) { return {a.s + b.s}; }
    __device__ static C get(const Acc& a) { return a.s; }
};

struct PolF32x2 {
    static constexpr bool factored = false;
    using S = float2;
    using C = df;
    using K = float2;
    static constexpr int kind = 2;
    __device__ static C ld(const S* p) {
        const float2 v = *p;
        return {v.x, v.y};
    }
    __device__ static void ld2(const S* p, C& a, C& b) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        a = {v.x, v.y};
        b = {v.z, v.w};
    }
    __device__ static C ldg(const S* p) {
        const float2 v = __ldg(p);
        return {v.x, v.y};
    }
    __device__ static void ld2p(const S* p, C& a, C& b) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a = {v.x, v.y};
        b = {v.z, v.w};
    }
    __device__ static void st(S* p, C v) { *p = make_float2(v.hi, v.lo); }
    __device__ static C add(C a, C b) { return df_add(a, b); }
    __device__ static C sub(C a, C b) { return df_add(a, {-b.hi, -b.lo}); }
    __device__ static C mul(C a, C b) { return df_mul(a, b); }
    __device__ static C zero() { return {0.f, 0.f}; }
    __device__ static C from_d(double x) {
        const float h = (float)x;
        return {h, (float)(x - (double)h)};
    }
    __host__ __device__ static double to_d(S x) { return (double)x.x + (double)x.y; }
    __device__ static bool sane(C v) { return fabsf(v.hi) < 1e30f; }
    __device__ static C shfl_xor(C v, int o) {
        return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    }
    // compensated dot product: s carries the running sum of the leading
    // products exactly up to the error e, which collects the two-sum and
    // two-product errors and the cross terms in FP32.
    struct Acc {
        float s, e;
    };
    __device__ static Acc acc0() { return {0.f, 0.f}; }
    // The running sum s and the error e each advance by one addition per
    // product; the two-sum error, the product error and the cross terms are
    // formed off that chain.
    __device__ static void fma(Acc& a, C x, C y) {
        const float p = x.hi * y.hi;
        const float pe = fmaf(x.hi, y.hi, -p);
        const df t = two_sum(a.s, p);
        const float c = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, t.lo + pe));
        a.s = t.hi;
        a.e = a.e + c;
    }
    __device__ static Acc merge(const Acc& a, const Acc& b) {
        const df t = two_sum(a.s, b.s);
        return {t.hi, (a.e + b.e) + t.lo};
    }
    __device__ static C get(const Acc& a) {
        const df t = two_sum(a.s, a.e);
        return t;
    }
};

struct PolF32F : PolF32 {
    static constexpr bool factored = true;
    static constexpr int kind = 3;
};

struct PolF32Fx2 : PolF32x2 {
    static constexpr bool factored = true;
    static constexpr int kind = 4;
    using K = float;
    // a += l x for a single-word factor element l: the two-float product
    // with its low word's cross term dropped (l has none)
    __device__ static void fma1(Acc& a, float l, C x) {
        const float p = l * x.hi;
        const float pe = fmaf(l, x.hi, -p);
        const df t = two_sum(a.s, p);
        a.s = t.hi;
        a.e = a.e + fmaf(l, x.lo, t.lo + pe);
    }
    __device__ static Acc shfl_xor_acc(const Acc& a, int o) {
        return {__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.e, o)};
    }
};

}  // namespace sfm
