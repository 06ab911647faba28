// 16-byte vector views of complex state blocks.
//
// complex64 blocks are read as float4 (two complex values per vector),
// complex128 blocks as double2 (one value).  A point row of ld complex values
// is SV = ld * sizeof(complex) / 16 vectors; all loads and stores of states
// are 128-bit.
#pragma once

#include <cuda_runtime.h>

namespace rsg {

template <typename R>
struct VT;

// Packed FP32x2 arithmetic (Blackwell): one instruction on two floats, with
// the same round-to-nearest result as two scalar operations.
union F2U {
    float2 f;
    unsigned long long u;
};
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    F2U x, y, z, d;
    x.f = a;
    y.f = b;
    z.f = c;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.u) : "l"(x.u), "l"(y.u), "l"(z.u));
    return d.f;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    F2U x, y, d;
    x.f = a;
    y.f = b;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.u) : "l"(x.u), "l"(y.u));
    return d.f;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    F2U x, y, d;
    x.f = a;
    y.f = b;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.u) : "l"(x.u), "l"(y.u));
    return d.f;
}

template <>
struct VT<float> {
    using T = float4;
    static constexpr int NC = 2;   // complex values per vector
    __device__ __forceinline__ static float2 lo(const T &a) { return make_float2(a.x, a.y); }
    __device__ __forceinline__ static float2 hi(const T &a) { return make_float2(a.z, a.w); }
    __device__ __forceinline__ static T join(float2 l, float2 h) { return make_float4(l.x, l.y, h.x, h.y); }
    __device__ __forceinline__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ static T ldg(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static void fma(T &acc, float w, const T &x) {
        const float2 ww = make_float2(w, w);
        acc = join(f2_fma(ww, lo(x), lo(acc)), f2_fma(ww, hi(x), hi(acc)));
    }
    __device__ __forceinline__ static T add(const T &a, const T &b) {
        return join(f2_add(lo(a), lo(b)), f2_add(hi(a), hi(b)));
    }
    __device__ __forceinline__ static T scale(float w, const T &a) {
        const float2 ww = make_float2(w, w);
        return join(f2_mul(ww, lo(a)), f2_mul(ww, hi(a)));
    }
    // (ar + i ai) * a, per complex component
    __device__ __forceinline__ static T cmul(float ar, float ai, const T &a) {
        return make_float4(ar * a.x - ai * a.y, ar * a.y + ai * a.x,
                           ar * a.z - ai * a.w, ar * a.w + ai * a.z);
    }
    // acc += (ar + i ai) * a
    __device__ __forceinline__ static void cfma(T &acc, float ar, float ai, const T &a) {
        acc.x = fmaf(ar, a.x, fmaf(-ai, a.y, acc.x));
        acc.y = fmaf(ar, a.y, fmaf(ai, a.x, acc.y));
        acc.z = fmaf(ar, a.z, fmaf(-ai, a.w, acc.z));
        acc.w = fmaf(ar, a.w, fmaf(ai, a.z, acc.w));
    }
    __device__ __forceinline__ static float comp(const T &a, int j) {
        return j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : a.w;
    }
};

template <>
struct VT<double> {
    using T = double2;
    static constexpr int NC = 1;
    __device__ __forceinline__ static T zero() { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ static T ldg(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static void fma(T &acc, double w, const T &x) {
        acc.x = fma_(w, x.x, acc.x);
        acc.y = fma_(w, x.y, acc.y);
    }
    __device__ __forceinline__ static double fma_(double a, double b, double c) {
        return ::fma(a, b, c);
    }
    __device__ __forceinline__ static T add(const T &a, const T &b) {
        return make_double2(a.x + b.x, a.y + b.y);
    }
    __device__ __forceinline__ static T scale(double w, const T &a) {
        return make_double2(w * a.x, w * a.y);
    }
    __device__ __forceinline__ static T cmul(double ar, double ai, const T &a) {
        return make_double2(ar * a.x - ai * a.y, ar * a.y + ai * a.x);
    }
    __device__ __forceinline__ static void cfma(T &acc, double ar, double ai, const T &a) {
        acc.x = ::fma(ar, a.x, ::fma(-ai, a.y, acc.x));
        acc.y = ::fma(ar, a.y, ::fma(ai, a.x, acc.y));
    }
    __device__ __forceinline__ static double comp(const T &a, int j) {
        return j == 0 ? a.x : a.y;
    }
};

}  // namespace rsg
