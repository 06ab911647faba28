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

template <>
struct VT<float> {
    using T = float4;
    static constexpr int NC = 2;   // complex values per vector
    __device__ __forceinline__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ static T ldg(const T *p) { return __ldg(p); }
    __device__ __forceinline__ static void fma(T &acc, float w, const T &x) {
        acc.x = fmaf(w, x.x, acc.x);
        acc.y = fmaf(w, x.y, acc.y);
        acc.z = fmaf(w, x.z, acc.z);
        acc.w = fmaf(w, x.w, acc.w);
    }
    __device__ __forceinline__ static T add(const T &a, const T &b) {
        return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
    __device__ __forceinline__ static T scale(float w, const T &a) {
        return make_float4(w * a.x, w * a.y, w * a.z, w * a.w);
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
