// Complex-scaled Hamiltonian (Sec. "Complex scaling and resonances"):
//
//   H_theta u = -1/2 e^{-2 i theta} lap u + v_theta u,
//
// the kinetic operator rotated by e^{-2 i theta} and the potential taken at
// the rotated coordinates, v_theta(r) = v(r e^{i theta}), which the caller
// supplies as one complex value per point.  H_theta is complex symmetric
// (u^T H_theta w = w^T H_theta u) but not Hermitian.
//
// k_apply_scaled: one thread per (point, 16-byte vector), the 25-point
// stencil with real weights summed over complex values and rotated once by
// (kr, ki) = (cos 2 theta, -sin 2 theta); the diagonal multiplies by the
// complex point value plus the real constant f0 (the shift of H - shift).
// The epilogue is the common one: out = alpha y (+ beta base), optional
// acc = acc_base + gamma out.  No projectors and no dipole field: the host
// refuses both while complex scaling is active.
#include <cmath>

#include "rsg_internal.h"
#include "rsg_odd.cuh"
#include "rsg_vec.cuh"

namespace rsg {

template <typename R>
__device__ __forceinline__ typename VT<R>::T scaled_value(const typename VT<R>::T *in, const Row &rw,
                                                          int x, int SV, int v) {
    if (x >= rw.xmin && x <= rw.xmax)
        return VT<R>::ldg(in + ((int64_t)rw.start + (x - rw.xmin)) * SV + v);
    return VT<R>::zero();
}

__device__ __forceinline__ Row scaled_row(const Row *rows, int y, int z, int ny, int nz) {
    if (y < 0 || y >= ny || z < 0 || z >= nz) return Row{0, 1, 0, 0};
    return rows[(int64_t)z * ny + y];
}

// ODD: the antisymmetric-image boundary of a box mesh (rsg_odd.cuh)
template <typename R, bool ODD>
__global__ void __launch_bounds__(256) k_apply_scaled(const ApplyArgs<R> a, const R *__restrict__ vt, R kr,
                                                      R ki) {
    using V = VT<R>;
    using T = typename V::T;
    const int row = blockIdx.x;
    const int ny = a.ny, nz = a.nz, SV = a.SV;
    const int y = row % ny, z = row / ny;
    const Row rc = a.rows[row];
    if (rc.xmin > rc.xmax) return;
    const T *__restrict__ in = (const T *)a.in;
    const int n = (rc.xmax - rc.xmin + 1) * SV;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int xo = t / SV, v = t - xo * SV;
        const int64_t idx = (int64_t)rc.start + xo;
        const int x = rc.xmin + xo;
        const T c = V::ldg(in + idx * SV + v);
        T lap = V::scale((R)3 * a.w[0], c);
        for (int k = 1; k <= 4; k++) {
            T s;
            if constexpr (ODD) {
                const int nx = a.nx;
                s = V::add(odd_site<R>(in, a.rows, x - k, y, z, nx, ny, nz, SV, v),
                           odd_site<R>(in, a.rows, x + k, y, z, nx, ny, nz, SV, v));
                s = V::add(s, odd_site<R>(in, a.rows, x, y - k, z, nx, ny, nz, SV, v));
                s = V::add(s, odd_site<R>(in, a.rows, x, y + k, z, nx, ny, nz, SV, v));
                s = V::add(s, odd_site<R>(in, a.rows, x, y, z - k, nx, ny, nz, SV, v));
                s = V::add(s, odd_site<R>(in, a.rows, x, y, z + k, nx, ny, nz, SV, v));
            } else {
                s = V::add(scaled_value<R>(in, rc, x - k, SV, v), scaled_value<R>(in, rc, x + k, SV, v));
                s = V::add(s, scaled_value<R>(in, scaled_row(a.rows, y - k, z, ny, nz), x, SV, v));
                s = V::add(s, scaled_value<R>(in, scaled_row(a.rows, y + k, z, ny, nz), x, SV, v));
                s = V::add(s, scaled_value<R>(in, scaled_row(a.rows, y, z - k, ny, nz), x, SV, v));
                s = V::add(s, scaled_value<R>(in, scaled_row(a.rows, y, z + k, ny, nz), x, SV, v));
            }
            V::fma(lap, a.w[k], s);
        }
        T acc = V::cmul(kr, ki, lap);
        const R vr = __ldg(vt + 2 * idx) + a.f0, vi = __ldg(vt + 2 * idx + 1);
        V::cfma(acc, vr, vi, c);
        const int64_t o = idx * SV + v;
        T y0 = V::cmul(a.ar, a.ai, acc);
        if (a.base != nullptr) V::cfma(y0, a.br, a.bi, ((const T *)a.base)[o]);
        ((T *)a.out)[o] = y0;
        if (a.acc != nullptr) {
            T s = a.acc_base != nullptr ? ((const T *)a.acc_base)[o] : ((T *)a.acc)[o];
            V::cfma(s, a.gr, a.gi, y0);
            ((T *)a.acc)[o] = s;
        }
    }
}

template <typename R>
cudaError_t launch_apply_scaled(const ApplyArgs<R> &a, const R *vt, double theta, cudaStream_t st) {
    if (a.ny * a.nz == 0) return cudaSuccess;
    k_apply_scaled<R, false>
        <<<a.ny * a.nz, 256, 0, st>>>(a, vt, (R)std::cos(2.0 * theta), (R)-std::sin(2.0 * theta));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_apply_scaled_odd(const ApplyArgs<R> &a, const R *vt, double theta, cudaStream_t st) {
    if (a.ny * a.nz == 0) return cudaSuccess;
    k_apply_scaled<R, true>
        <<<a.ny * a.nz, 256, 0, st>>>(a, vt, (R)std::cos(2.0 * theta), (R)-std::sin(2.0 * theta));
    return cudaGetLastError();
}

template cudaError_t launch_apply_scaled<float>(const ApplyArgs<float> &, const float *, double, cudaStream_t);
template cudaError_t launch_apply_scaled<double>(const ApplyArgs<double> &, const double *, double, cudaStream_t);
template cudaError_t launch_apply_scaled_odd<float>(const ApplyArgs<float> &, const float *, double, cudaStream_t);
template cudaError_t launch_apply_scaled_odd<double>(const ApplyArgs<double> &, const double *, double,
                                                     cudaStream_t);

}  // namespace rsg
