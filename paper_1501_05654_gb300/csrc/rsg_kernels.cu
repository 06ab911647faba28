// Hamiltonian application kernels.
//
// H u = -1/2 lap u + (V + eps dir.r) u + sum_a sum_ij |p_ai> h_a,ij <p_aj|u>
// on a uniform mesh stored as rows of contiguous points (z slowest, x
// fastest), with the 8th-order 25-point star Laplacian (radius 4 per axis)
// and zero values outside the mesh (arXiv:1501.05654, Sec. 1: high-order
// finite differences on a real-space grid; Sec. "Performance": Hamiltonian
// application on a group of states, fields as linear arrays plus grid
// tables).
//
// The result goes through one epilogue shared by every caller:
//     y = alpha * (H u) [+ beta * base];  out = y;  [acc += gamma * y]
// which is a Horner stage of the Taylor-4 exponential (alpha = -i tau/k,
// base = psi), a plain application (alpha = 1), or one explicit power of
// A = -i tau H with the running Taylor sum in acc.
//
// Kernels:
//   k_apply_zmarch  each thread owns RX consecutive x points of one row and
//                   one 16-byte state vector and marches along z, keeping the
//                   nine z-neighbours in registers; x/y neighbours come
//                   through L1.  Projector terms are added in the epilogue
//                   through a per-point CSR list of sphere entries.
//   k_apply_naive   one thread per (point, vector), all 25 neighbours loaded;
//                   the plain reference GPU path.
//   k_proj_dot      partial sums of <p_ai|u_s> over sphere chunks (FP32
//                   products and partial sums for complex64, FP64 across
//                   chunks), k_proj_reduce: h^3 sum over chunks, times h_a.
#include "rsg_internal.h"
#include "rsg_vec.cuh"

namespace rsg {

// ------------------------------------------------------------ epilogue ---
template <typename R>
__device__ __forceinline__ void finish_point(const ApplyArgs<R> &a, int64_t idx, int x, int y,
                                             int z, int v,
                                             const typename VT<R>::T &center,
                                             typename VT<R>::T acc) {
    using V = VT<R>;
    using T = typename V::T;
    const int SV = a.SV;
    R diag = a.V[idx] + a.f0 + a.fx * (R)x + a.fy * (R)y + a.fz * (R)z;
    V::fma(acc, diag, center);
    if (a.nl_ptr != nullptr) {
        const int e0 = a.nl_ptr[idx], e1 = a.nl_ptr[idx + 1];
        const T *D = (const T *)a.D;
        for (int e = e0; e < e1; e++) {
            const int q = a.nl_ent[e];
            const int at = a.q_atom[q];
            const R *pv = a.q_p + (int64_t)q * a.npmax;
            const T *Da = D + (int64_t)at * a.npmax * SV + v;
            for (int i = 0; i < a.npmax; i++) V::fma(acc, pv[i], Da[(int64_t)i * SV]);
        }
    }
    const int64_t o = idx * SV + v;
    T y0 = V::cmul(a.ar, a.ai, acc);
    if (a.base != nullptr) V::cfma(y0, a.br, a.bi, ((const T *)a.base)[o]);
    ((T *)a.out)[o] = y0;
    if (a.acc != nullptr) {
        T s = ((T *)a.acc)[o];
        V::cfma(s, a.gr, a.gi, y0);
        ((T *)a.acc)[o] = s;
    }
}

// Value of vector v at bbox (x, row) or zero outside the mesh.
template <typename R>
__device__ __forceinline__ typename VT<R>::T row_value(const typename VT<R>::T *in,
                                                       const Row &rw, int x, int SV, int v) {
    if (x >= rw.xmin && x <= rw.xmax)
        return VT<R>::ldg(in + ((int64_t)rw.start + (x - rw.xmin)) * SV + v);
    return VT<R>::zero();
}

__device__ __forceinline__ Row load_row(const Row *rows, int y, int z, int ny, int nz) {
    if (y < 0 || y >= ny || z < 0 || z >= nz) return Row{0, 1, 0, 0};
    return rows[(int64_t)z * ny + y];
}

// --------------------------------------------------------- z-marching ---
template <typename R, int RX>
__global__ void __launch_bounds__(256) k_apply_zmarch(const ApplyArgs<R> a) {
    using V = VT<R>;
    using T = typename V::T;
    const Tile tl = a.tiles[blockIdx.x];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    if (v >= a.SV) return;
    const int x0 = (tl.tx * blockDim.y + threadIdx.y) * RX;
    const int y = tl.ty * blockDim.z + threadIdx.z;
    if (y >= a.ny || x0 >= a.nx) return;
    const T *__restrict__ in = (const T *)a.in;
    const int SV = a.SV, ny = a.ny, nz = a.nz;
    const R w0 = a.w[0], w1 = a.w[1], w2 = a.w[2], w3 = a.w[3], w4 = a.w[4];
    const R wk[5] = {w0, w1, w2, w3, w4};

    T ring[9][RX];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const Row rw = load_row(a.rows, y, tl.zlo - 4 + k, ny, nz);
#pragma unroll
        for (int r = 0; r < RX; r++) ring[k][r] = row_value<R>(in, rw, x0 + r, SV, v);
    }
    for (int z = tl.zlo; z < tl.zhi; z++) {
        {
            const Row rw = load_row(a.rows, y, z + 4, ny, nz);
#pragma unroll
            for (int r = 0; r < RX; r++) ring[8][r] = row_value<R>(in, rw, x0 + r, SV, v);
        }
        const Row rc = load_row(a.rows, y, z, ny, nz);
        if (x0 + RX - 1 >= rc.xmin && x0 <= rc.xmax) {
            T acc[RX];
#pragma unroll
            for (int r = 0; r < RX; r++) {
                acc[r] = V::scale((R)3 * w0, ring[4][r]);
#pragma unroll
                for (int k = 1; k <= 4; k++) V::fma(acc[r], wk[k], V::add(ring[4 - k][r], ring[4 + k][r]));
            }
            // x neighbours: inside the run from the ring, outside from L1
            T xl[4], xr[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                xl[k] = row_value<R>(in, rc, x0 - 1 - k, SV, v);
                xr[k] = row_value<R>(in, rc, x0 + RX + k, SV, v);
            }
#pragma unroll
            for (int r = 0; r < RX; r++) {
#pragma unroll
                for (int k = 1; k <= 4; k++) {
                    const T left = (r - k >= 0) ? ring[4][(r - k) >= 0 ? r - k : 0] : xl[k - r - 1 >= 0 ? k - r - 1 : 0];
                    const T right = (r + k < RX) ? ring[4][(r + k) < RX ? r + k : 0] : xr[(r + k - RX) >= 0 ? r + k - RX : 0];
                    V::fma(acc[r], wk[k], V::add(left, right));
                }
            }
            // y neighbours
#pragma unroll
            for (int k = 1; k <= 4; k++) {
                const Row ra = load_row(a.rows, y - k, z, ny, nz);
                const Row rb = load_row(a.rows, y + k, z, ny, nz);
#pragma unroll
                for (int r = 0; r < RX; r++)
                    V::fma(acc[r], wk[k], V::add(row_value<R>(in, ra, x0 + r, SV, v),
                                                 row_value<R>(in, rb, x0 + r, SV, v)));
            }
#pragma unroll
            for (int r = 0; r < RX; r++) {
                const int x = x0 + r;
                if (x >= rc.xmin && x <= rc.xmax) {
                    const int64_t idx = (int64_t)rc.start + (x - rc.xmin);
                    finish_point<R>(a, idx, x, y, z, v, ring[4][r], acc[r]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++)
#pragma unroll
            for (int r = 0; r < RX; r++) ring[k][r] = ring[k + 1][r];
    }
}

// --------------------------------------------------------------- naive ---
template <typename R>
__global__ void __launch_bounds__(256) k_apply_naive(const ApplyArgs<R> a) {
    using V = VT<R>;
    using T = typename V::T;
    const int row = blockIdx.x;
    const int ny = a.ny, nz = a.nz, SV = a.SV;
    const int y = row % ny, z = row / ny;
    const Row rc = a.rows[row];
    if (rc.xmin > rc.xmax) return;
    const T *__restrict__ in = (const T *)a.in;
    const int64_t n = (int64_t)(rc.xmax - rc.xmin + 1) * SV;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const int xo = (int)(t / SV), v = (int)(t % SV);
        const int x = rc.xmin + xo;
        const int64_t idx = (int64_t)rc.start + xo;
        const T c = V::ldg(in + idx * SV + v);
        T acc = V::scale((R)3 * a.w[0], c);
        for (int k = 1; k <= 4; k++) {
            T s = V::add(row_value<R>(in, rc, x - k, SV, v), row_value<R>(in, rc, x + k, SV, v));
            s = V::add(s, row_value<R>(in, load_row(a.rows, y - k, z, ny, nz), x, SV, v));
            s = V::add(s, row_value<R>(in, load_row(a.rows, y + k, z, ny, nz), x, SV, v));
            s = V::add(s, row_value<R>(in, load_row(a.rows, y, z - k, ny, nz), x, SV, v));
            s = V::add(s, row_value<R>(in, load_row(a.rows, y, z + k, ny, nz), x, SV, v));
            V::fma(acc, a.w[k], s);
        }
        finish_point<R>(a, idx, x, y, z, v, c, acc);
    }
}

static inline int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <typename R>
cudaError_t launch_apply(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st) {
    if (cfg.kernel == 1) {
        k_apply_naive<R><<<a.ny * a.nz, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    const int cv = pow2_at_least(a.SV) < 8 ? pow2_at_least(a.SV) : 8;
    int ty = cfg.ty;
    while (cv * ty > 256) ty >>= 1;
    const int nxr = 256 / (cv * ty);
    dim3 block(cv, nxr, ty);
    dim3 grid(ntiles, (a.SV + cv - 1) / cv);
    if (ntiles == 0) return cudaSuccess;
    switch (cfg.rx) {
    case 1: k_apply_zmarch<R, 1><<<grid, block, 0, st>>>(a); break;
    case 2: k_apply_zmarch<R, 2><<<grid, block, 0, st>>>(a); break;
    default: k_apply_zmarch<R, 4><<<grid, block, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------- projectors ---
// Block: (BV vectors) x (PL point lanes).  Chunk c covers entries [q0, q1)
// of one atom.  partial[((c * npmax + i) * SV + v) * 2 * NC + comp] (FP64).
template <typename R, int NP>
__global__ void __launch_bounds__(256) k_proj_dot(const typename VT<R>::T *__restrict__ u, int SV,
                                                  const int32_t *__restrict__ q_pt,
                                                  const R *__restrict__ q_p,
                                                  const int32_t *__restrict__ chunk_q0,
                                                  const int32_t *__restrict__ chunk_q1,
                                                  double *__restrict__ partial) {
    using V = VT<R>;
    using T = typename V::T;
    constexpr int NCOMP = 2 * V::NC;
    __shared__ double red[256 * NCOMP];
    const int c = blockIdx.x;
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    const int q0 = chunk_q0[c], q1 = chunk_q1[c];
    T acc[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) acc[i] = V::zero();
    if (v < SV) {
        for (int q = q0 + threadIdx.y; q < q1; q += blockDim.y) {
            const T val = V::ldg(u + (int64_t)q_pt[q] * SV + v);
#pragma unroll
            for (int i = 0; i < NP; i++) V::fma(acc[i], q_p[(int64_t)q * NP + i], val);
        }
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i = 0; i < NP; i++) {
#pragma unroll
        for (int j = 0; j < NCOMP; j++) red[tid * NCOMP + j] = (double)V::comp(acc[i], j);
        __syncthreads();
        if (threadIdx.y == 0 && v < SV) {
            double s[NCOMP];
#pragma unroll
            for (int j = 0; j < NCOMP; j++) s[j] = 0.0;
            for (int l = 0; l < (int)blockDim.y; l++)
#pragma unroll
                for (int j = 0; j < NCOMP; j++) s[j] += red[(l * blockDim.x + threadIdx.x) * NCOMP + j];
            double *dst = partial + (((int64_t)c * NP + i) * SV + v) * NCOMP;
#pragma unroll
            for (int j = 0; j < NCOMP; j++) dst[j] = s[j];
        }
        __syncthreads();
    }
}

template <typename R>
cudaError_t launch_proj_dot(const void *u, int SV, const ProjDev &pj, double *partial,
                            cudaStream_t st) {
    if (pj.natoms == 0 || pj.nchunks == 0) return cudaSuccess;
    const int bv = SV < 32 ? SV : 32;
    const int pl = 256 / bv > 64 ? 64 : 256 / bv;
    dim3 block(bv, pl);
    dim3 grid(pj.nchunks, (SV + bv - 1) / bv);
    using T = typename VT<R>::T;
    const T *uu = (const T *)u;
    const R *qp = (const R *)pj.q_p;
    switch (pj.npmax) {
    case 1: k_proj_dot<R, 1><<<grid, block, 0, st>>>(uu, SV, pj.q_pt, qp, pj.chunk_q0, pj.chunk_q1, partial); break;
    case 4: k_proj_dot<R, 4><<<grid, block, 0, st>>>(uu, SV, pj.q_pt, qp, pj.chunk_q0, pj.chunk_q1, partial); break;
    case 9: k_proj_dot<R, 9><<<grid, block, 0, st>>>(uu, SV, pj.q_pt, qp, pj.chunk_q0, pj.chunk_q1, partial); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// One thread per (atom, complex column s).  c_i = h3 * sum over the atom's
// chunks; D[a, i, s] = sum_j h_a[i][j] c_j, stored in the compute type.
template <typename R>
__global__ void k_proj_reduce(const double *__restrict__ partial, int SV, int natoms, int npmax,
                              const int32_t *__restrict__ atom_chunk0,
                              const double *__restrict__ hm, double h3, R *__restrict__ D) {
    constexpr int NC = VT<R>::NC;
    const int ldc = SV * NC;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= natoms * ldc) return;
    const int a = t / ldc, s = t % ldc;
    double cr[9], ci[9];
    for (int i = 0; i < npmax; i++) {
        double sr = 0.0, si = 0.0;
        for (int c = atom_chunk0[a]; c < atom_chunk0[a + 1]; c++) {
            const double *p = partial + (((int64_t)c * npmax + i) * ldc + s) * 2;
            sr += p[0];
            si += p[1];
        }
        cr[i] = h3 * sr;
        ci[i] = h3 * si;
    }
    for (int i = 0; i < npmax; i++) {
        double dr = 0.0, di = 0.0;
        for (int j = 0; j < npmax; j++) {
            const double hij = hm[((int64_t)a * npmax + i) * npmax + j];
            dr += hij * cr[j];
            di += hij * ci[j];
        }
        R *dst = D + (((int64_t)a * npmax + i) * ldc + s) * 2;
        dst[0] = (R)dr;
        dst[1] = (R)di;
    }
}

template <typename R>
cudaError_t launch_proj_reduce(const double *partial, int SV, const ProjDev &pj, double h3,
                               void *D, cudaStream_t st) {
    if (pj.natoms == 0) return cudaSuccess;
    const int n = pj.natoms * SV * VT<R>::NC;
    k_proj_reduce<R><<<(n + 127) / 128, 128, 0, st>>>(partial, SV, pj.natoms, pj.npmax,
                                                       pj.atom_chunk0, pj.hm, h3, (R *)D);
    return cudaGetLastError();
}

template cudaError_t launch_apply<float>(const ApplyArgs<float> &, const TileCfg &, int, cudaStream_t);
template cudaError_t launch_apply<double>(const ApplyArgs<double> &, const TileCfg &, int, cudaStream_t);
template cudaError_t launch_proj_dot<float>(const void *, int, const ProjDev &, double *, cudaStream_t);
template cudaError_t launch_proj_dot<double>(const void *, int, const ProjDev &, double *, cudaStream_t);
template cudaError_t launch_proj_reduce<float>(const double *, int, const ProjDev &, double, void *, cudaStream_t);
template cudaError_t launch_proj_reduce<double>(const double *, int, const ProjDev &, double, void *, cudaStream_t);

}  // namespace rsg
