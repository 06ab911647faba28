// Hamiltonian application kernels.
//
// H u = -1/2 lap u + (V + eps dir.r) u + sum_a sum_ij |p_ai> h_a,ij <p_aj|u>
// on a uniform mesh stored as rows of contiguous points (z slowest, x
// fastest), with the 8th-order 25-point star Laplacian (radius 4 per axis)
// and zero values outside the mesh (arXiv:1501.05654, Sec. 1: high-order
// finite differences on a real-space grid; Sec. "Parallelization, optimizations and graphics processing units": Hamiltonian
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
#include <cuda.h>

#include "rsg_async.cuh"
#include "rsg_batch.cuh"
#include "rsg_internal.h"
#include "rsg_odd.cuh"
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
    if (a.twocol) {
        // two columns with their own field terms: column (v, component
        // pair) of a complex64 vector, or vector v of complex128
        auto diag_of = [&](int c) {
            return a.V[idx] + a.cf[c][0] + a.cf[c][1] * (R)x + a.cf[c][2] * (R)y + a.cf[c][3] * (R)z;
        };
        if constexpr (sizeof(R) == 4) {
            const R d0 = diag_of(0), d1 = diag_of(1);
            acc.x = fmaf(d0, center.x, acc.x);
            acc.y = fmaf(d0, center.y, acc.y);
            acc.z = fmaf(d1, center.z, acc.z);
            acc.w = fmaf(d1, center.w, acc.w);
        } else {
            V::fma(acc, diag_of(v), center);
        }
    } else {
        const R diag = a.V[idx] + a.f0 + a.fx * (R)x + a.fy * (R)y + a.fz * (R)z;
        V::fma(acc, diag, center);
    }
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
    T y0;
    if (a.twocol) {
        if constexpr (sizeof(R) == 4) {
            const R r0 = a.ca[0][0], i0 = a.ca[0][1], r1 = a.ca[1][0], i1 = a.ca[1][1];
            y0 = make_float4(r0 * acc.x - i0 * acc.y, r0 * acc.y + i0 * acc.x, r1 * acc.z - i1 * acc.w,
                             r1 * acc.w + i1 * acc.z);
        } else {
            y0 = V::cmul(a.ca[v][0], a.ca[v][1], acc);
        }
    } else {
        y0 = V::cmul(a.ar, a.ai, acc);
    }
    if (a.base != nullptr) V::cfma(y0, a.br, a.bi, ((const T *)a.base)[o]);
    ((T *)a.out)[o] = y0;
    if (a.acc != nullptr) {
        T s = a.acc_base != nullptr ? ((const T *)a.acc_base)[o] : ((T *)a.acc)[o];
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
constexpr int kMaxTY = 16, kMaxZseg = 120;
constexpr int kSRows = (kMaxTY + 8) * (kMaxZseg + 8);

// Branch-free read of vector v at bbox x of a row: out-of-row lanes load a
// valid dummy address (point 0) and select zero, so every load of an
// iteration can be in flight at once.
template <typename R>
__device__ __forceinline__ typename VT<R>::T srow_value(const typename VT<R>::T *in, const SRow &rw,
                                                        int x, int SV, int v) {
    const bool ok = (x >= rw.xmin) & (x <= rw.xmax);
    const int64_t idx = ok ? (int64_t)rw.start + (x - rw.xmin) : 0;
    const typename VT<R>::T val = VT<R>::ldg(in + idx * SV + v);
    return ok ? val : VT<R>::zero();
}

template <typename R, int RX>
__global__ void __launch_bounds__(256, (RX <= 2 ? 2 : 1)) k_apply_zmarch(const ApplyArgs<R> a) {
    using V = VT<R>;
    using T = typename V::T;
    __shared__ SRow srows[kSRows];
    const Tile tl = a.tiles[blockIdx.x];
    const int ny = a.ny, nz = a.nz, SV = a.SV;
    const int TY = blockDim.z;
    const int ybase = tl.ty * TY - 4, zbase = tl.zlo - 4;
    const int nyr = TY + 8, nzr = tl.zhi - tl.zlo + 8;
    // stage the rows this block touches: y in [ybase, ybase+nyr), z in [zbase, zbase+nzr)
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    for (int i = tid; i < nyr * nzr; i += nthr) {
        const int yy = ybase + i % nyr, zz = zbase + i / nyr;
        SRow r{0, 1, 0};
        if (yy >= 0 && yy < ny && zz >= 0 && zz < nz) {
            const Row g = a.rows[(int64_t)zz * ny + yy];
            r.start = g.start;
            r.xmin = (int16_t)g.xmin;
            r.xmax = (int16_t)g.xmax;
        }
        srows[i] = r;
    }
    __syncthreads();
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    if (v >= SV) return;
    const int x0 = (tl.tx * blockDim.y + threadIdx.y) * RX;
    const int y = tl.ty * TY + threadIdx.z;
    if (y >= ny || x0 >= a.nx) return;
    const T *__restrict__ in = (const T *)a.in;
    const R wk[5] = {a.w[0], a.w[1], a.w[2], a.w[3], a.w[4]};
    const int yo = threadIdx.z + 4;   // own row offset in the staged table
    auto srow = [&](int dy, int z) -> const SRow & { return srows[(z - zbase) * nyr + yo + dy]; };

    T ring[9][RX];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const SRow rw = srow(0, tl.zlo - 4 + k);
#pragma unroll
        for (int r = 0; r < RX; r++) ring[k][r] = srow_value<R>(in, rw, x0 + r, SV, v);
    }
    for (int z = tl.zlo; z < tl.zhi; z++) {
        {
            const SRow rw = srow(0, z + 4);
#pragma unroll
            for (int r = 0; r < RX; r++) ring[8][r] = srow_value<R>(in, rw, x0 + r, SV, v);
        }
        const SRow rc = srow(0, z);
        if (x0 + RX - 1 >= rc.xmin && x0 <= rc.xmax) {
            T acc[RX];
#pragma unroll
            for (int r = 0; r < RX; r++) {
                acc[r] = V::scale((R)3 * wk[0], ring[4][r]);
#pragma unroll
                for (int k = 1; k <= 4; k++) V::fma(acc[r], wk[k], V::add(ring[4 - k][r], ring[4 + k][r]));
            }
            // x neighbours: inside the run from the ring, outside from L1
#pragma unroll
            for (int k = 1; k <= 4; k++) {
#pragma unroll
                for (int r = 0; r < RX; r++) {
                    const T left = (r - k >= 0) ? ring[4][(r - k) >= 0 ? r - k : 0]
                                                : srow_value<R>(in, rc, x0 + r - k, SV, v);
                    const T right = (r + k < RX) ? ring[4][(r + k) < RX ? r + k : 0]
                                                 : srow_value<R>(in, rc, x0 + r + k, SV, v);
                    V::fma(acc[r], wk[k], V::add(left, right));
                }
            }
            // y neighbours
#pragma unroll
            for (int k = 1; k <= 4; k++) {
                const SRow ra = srow(-k, z), rb = srow(k, z);
#pragma unroll
                for (int r = 0; r < RX; r++)
                    V::fma(acc[r], wk[k], V::add(srow_value<R>(in, ra, x0 + r, SV, v),
                                                 srow_value<R>(in, rb, x0 + r, SV, v)));
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

// ------------------------------------------------- shared-memory staged ---
// k_apply_staged: a block owns a TX x TY tile of one state chunk (CV 16-byte
// vectors per point) and streams the planes z = zlo-4 .. zhi+3 of the tile
// plus a 4-point halo in x and y through an NS-deep ring of shared-memory
// slots filled with cp.async (ghost points are zero-filled by the copy).
// When plane p has landed, every thread adds plane p's contributions to a
// register queue of nine pending outputs p-4 .. p+4 (z part: w_|k| c_p to
// output p+k; x/y part and the diagonal to output p), then retires output
// p-4 through the epilogue.  The queue rotates by renaming (the plane loop
// is unrolled nine times), so no values move between registers.  Each state
// value crosses L2 -> shared memory once per tile (plus the halo); all
// neighbour reads are fixed-offset shared-memory loads; all offsets are
// 32-bit (the host checks P * SV < 2^31).
// Epilogue of the staged kernel: y = alpha * acc + beta * base (base already
// in registers), out = y, optional acc += gamma * y.  Projector terms are
// added afterwards by k_proj_scatter.
template <typename R>
__device__ __forceinline__ void finish_staged(const ApplyArgs<R> &a, int o, typename VT<R>::T acc,
                                              const typename VT<R>::T &base) {
    using V = VT<R>;
    using T = typename V::T;
    T y0 = V::cmul(a.ar, a.ai, acc);
    if (a.base != nullptr) V::cfma(y0, a.br, a.bi, base);
    ((T *)a.out)[o] = y0;
    if (a.acc != nullptr) {
        T s = a.acc_base != nullptr ? ((const T *)a.acc_base)[o] : ((T *)a.acc)[o];
        V::cfma(s, a.gr, a.gi, y0);
        ((T *)a.acc)[o] = s;
    }
}

// Fixed geometry of the staged kernel: NT threads = CV vectors x TX
// columns x 16 rows, one point per thread along x; every shared-memory offset
// is then a compile-time constant.
template <int CV, int NT = 512>
struct StagedGeom {
    static constexpr int TY = 16, TX = NT / 16 / CV, WX = TX + 8, WY = TY + 8, NTHR = NT;
    // the star stencil reads a cross: the TY middle rows at full width and
    // four rows above and below at the interior width; corners are not staged
    static constexpr int NMID = TY * WX, NCROSS = NMID + 8 * TX, SLOT = WY * WX * CV;
};

template <typename R, int CV, int NT>
struct StageCtx {
    using T = typename VT<R>::T;
    const ApplyArgs<R> *a;
    const SRow *srows;
    const T *slots;
    const T *bslots;     // per thread: base of its output, NS slots x 512
    const R *vslots;     // per thread: V of its column, NS slots x 512
    int tid;
    int xr, yi, cv, v, y, x0;    // thread's tile coordinates and global x
    int zbase, zlo, zhi;
    int zc0, zc1;                // planes where the thread's column has points
    R w0, w1, w2, w3, w4;
};

// Plane j has landed in its slot: add its contributions, retire output p-4.
// Queue slot of output p + (k - 4) is (k + PH) % 9.
template <typename R, int CV, int NT, int NS, int PH>
__device__ __forceinline__ void stage_plane(const StageCtx<R, CV, NT> &c, int j, typename VT<R>::T (&q)[9]) {
    using V = VT<R>;
    using T = typename V::T;
    using G = StagedGeom<CV, NT>;
    constexpr int Q0 = (0 + PH) % 9, Q1 = (1 + PH) % 9, Q2 = (2 + PH) % 9, Q3 = (3 + PH) % 9;
    constexpr int Q4 = (4 + PH) % 9, Q5 = (5 + PH) % 9, Q6 = (6 + PH) % 9, Q7 = (7 + PH) % 9;
    constexpr int Q8 = (8 + PH) % 9;
    constexpr int RS = G::WX * CV;     // one slot row
    const ApplyArgs<R> &a = *c.a;
    const T *sl = c.slots + (j % NS) * G::SLOT;
    const int p = c.zbase + j;
    const T *cp = sl + ((c.yi + 4) * G::WX + c.xr + 4) * CV + c.cv;
    // a column off the mesh at plane p contributes nothing (its values and
    // outputs there are zero / absent): skip the arithmetic
    if (p >= c.zc0 && p <= c.zc1) {
        const T cval = cp[0];
        V::fma(q[Q3], c.w1, cval);
        V::fma(q[Q5], c.w1, cval);
        V::fma(q[Q2], c.w2, cval);
        V::fma(q[Q6], c.w2, cval);
        V::fma(q[Q1], c.w3, cval);
        V::fma(q[Q7], c.w3, cval);
        V::fma(q[Q0], c.w4, cval);
        V::fma(q[Q8], c.w4, cval);
        T s = V::scale((R)3 * c.w0, cval);
        V::fma(s, c.w1, V::add(V::add(cp[-CV], cp[CV]), V::add(cp[-RS], cp[RS])));
        V::fma(s, c.w2, V::add(V::add(cp[-2 * CV], cp[2 * CV]), V::add(cp[-2 * RS], cp[2 * RS])));
        V::fma(s, c.w3, V::add(V::add(cp[-3 * CV], cp[3 * CV]), V::add(cp[-3 * RS], cp[3 * RS])));
        V::fma(s, c.w4, V::add(V::add(cp[-4 * CV], cp[4 * CV]), V::add(cp[-4 * RS], cp[4 * RS])));
        // diagonal: staged V (zero outside the mesh, where c is zero too)
        const R diag = c.vslots[(j % NS) * G::NTHR + c.tid] + a.f0 + a.fx * (R)c.x0 + a.fy * (R)c.y +
                       a.fz * (R)p;
        V::fma(s, diag, cval);
        q[Q4] = V::add(q[Q4], s);
    }
    const int zo = p - 4;
    if (zo >= c.zlo && zo < c.zhi && c.v < a.SV) {
        const SRow ro = c.srows[(j - 4) * G::WY + c.yi + 4];
        const int x = c.x0;
        if (x >= ro.xmin && x <= ro.xmax) {
            const int idx = ro.start + (x - ro.xmin);
            finish_staged<R>(a, idx * a.SV + c.v, q[Q0], c.bslots[(j % NS) * G::NTHR + c.tid]);
        }
    }
    q[Q0] = V::zero();
}

// One block of the staged kernel: tile tl, state chunk `chunk` of the
// system described by a.
template <typename R, int CV, int NS, int NT = 512>
__device__ __forceinline__ void staged_block(const ApplyArgs<R> &a, const Tile tl, const int chunk,
                                             unsigned char *smraw, SRow *srows) {
    using V = VT<R>;
    using T = typename V::T;
    using G = StagedGeom<CV, NT>;
    constexpr int TX = G::TX, TY = G::TY, WX = G::WX, WY = G::WY;
    const int ny = a.ny, nz = a.nz, SV = a.SV;
    const int xbase = tl.tx * TX - 4, ybase = tl.ty * TY - 4, zbase = tl.zlo - 4;
    const int nzr = tl.zhi - tl.zlo + 8;
    const int tid = (threadIdx.z * TX + threadIdx.y) * CV + threadIdx.x;
    for (int i = tid; i < WY * nzr; i += G::NTHR) {
        const int zz = i / WY;
        const int yy = ybase + (i - zz * WY);
        const int zg = zbase + zz;
        SRow r{0, 1, 0};
        if (yy >= 0 && yy < ny && zg >= 0 && zg < nz) {
            const Row g = a.rows[zg * ny + yy];
            r.start = g.start;
            r.xmin = (int16_t)g.xmin;
            r.xmax = (int16_t)g.xmax;
        }
        srows[i] = r;
    }
    __syncthreads();
    T *slots = (T *)smraw;
    T *bslots = slots + NS * G::SLOT;                          // NS x 512
    R *vslots = (R *)(bslots + NS * G::NTHR);                  // NS x 512
    const T *__restrict__ in = (const T *)a.in;
    const int cvl = threadIdx.x;
    const int v = chunk * CV + cvl;
    const bool vok = v < SV;
    const int yown = threadIdx.z + 4;
    const int xown = tl.tx * TX + threadIdx.y;
    const unsigned bsh = (unsigned)__cvta_generic_to_shared(bslots);
    const unsigned vsh = (unsigned)__cvta_generic_to_shared(vslots);
    const T *__restrict__ basep = (const T *)a.base;
    // own-point data that travels with plane j: V at plane j (diagonal on
    // arrival) and the base value of the output retired at plane j (j - 4)
    auto stage_epi = [&](int j) {
        const int sl = j % NS;
        const SRow rj = srows[j * WY + yown];
        const bool okj = (xown >= rj.xmin) & (xown <= rj.xmax);
        cp_async_small<sizeof(R)>(vsh + (unsigned)((sl * G::NTHR + tid) * sizeof(R)),
                                  a.V + (okj ? rj.start + (xown - rj.xmin) : 0), okj ? (int)sizeof(R) : 0);
        if (basep != nullptr && j >= 4) {
            const SRow ro = srows[(j - 4) * WY + yown];
            const bool ok = (xown >= ro.xmin) & (xown <= ro.xmax) & vok;
            const int o = ok ? (ro.start + (xown - ro.xmin)) * SV + v : 0;
            cp_async16(bsh + (unsigned)((sl * G::NTHR + tid) * 16), basep + o, ok ? 16 : 0);
        }
    };

    // staging assignment: this thread copies cross points pi = tid / CV + m * STEP
    constexpr int STEP = G::NTHR / CV;
    const int pi0 = tid / CV;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(slots);
    auto stage = [&](int j) {
        stage_epi(j);
        const unsigned dst0 = sbase + (unsigned)(((j % NS) * G::SLOT + cvl) * 16);
        const SRow *rr = srows + j * WY;
#pragma unroll
        for (int m = 0; m < (G::NCROSS + STEP - 1) / STEP; m++) {
            const int pi = pi0 + m * STEP;
            if (pi < G::NCROSS) {
                int yy, xx;
                if (pi < G::NMID) {
                    yy = 4 + pi / WX;
                    xx = pi - (yy - 4) * WX;
                } else {
                    const int e = pi - G::NMID, r = e / TX;
                    yy = r < 4 ? r : TY + r;
                    xx = 4 + (e - r * TX);
                }
                const SRow rw = rr[yy];
                const int x = xbase + xx;
                const bool ok = (x >= rw.xmin) & (x <= rw.xmax) & vok;
                const int off = ok ? (rw.start + (x - rw.xmin)) * SV + v : 0;
                cp_async16(dst0 + (unsigned)((yy * WX + xx) * CV * 16), in + off, ok ? 16 : 0);
            }
        }
    };

    StageCtx<R, CV, NT> c;
    c.a = &a;
    c.srows = srows;
    c.slots = slots;
    c.bslots = bslots;
    c.vslots = vslots;
    c.tid = tid;
    c.xr = threadIdx.y;
    c.yi = threadIdx.z;
    c.cv = cvl;
    c.v = v;
    c.y = tl.ty * TY + threadIdx.z;
    c.x0 = xown;
    c.zbase = zbase;
    c.zlo = tl.zlo;
    c.zhi = tl.zhi;
    c.w0 = a.w[0];
    c.w1 = a.w[1];
    c.w2 = a.w[2];
    c.w3 = a.w[3];
    c.w4 = a.w[4];
    T q[9];
#pragma unroll
    for (int k = 0; k < 9; k++) q[k] = V::zero();

    const int np = nzr;
    // column z-range of this thread (the mesh meets each column in one run)
    c.zc0 = 1 << 30;
    c.zc1 = -(1 << 30);
    for (int jj = 0; jj < np; jj++) {
        const SRow rw = srows[jj * WY + yown];
        if (xown >= rw.xmin && xown <= rw.xmax) {
            c.zc0 = min(c.zc0, zbase + jj);
            c.zc1 = max(c.zc1, zbase + jj);
        }
    }
#pragma unroll 1
    for (int j = 0; j < NS - 1; j++) {
        if (j < np) stage(j);
        cp_async_commit();
    }
    // plane j has landed for every thread after the barrier; the slot then
    // refilled (plane j + NS - 1) was last read at plane j - 1, which every
    // thread finished before reaching the barrier: one barrier per plane
    auto pre = [&](int j) {
        cp_async_wait<NS - 2>();
        __syncthreads();
        if (j + NS - 1 < np) stage(j + NS - 1);
        cp_async_commit();
    };
    int j = 0;
#pragma unroll 1
    for (; j + 9 <= np; j += 9) {
        pre(j + 0); stage_plane<R, CV, NT, NS, 0>(c, j + 0, q);
        pre(j + 1); stage_plane<R, CV, NT, NS, 1>(c, j + 1, q);
        pre(j + 2); stage_plane<R, CV, NT, NS, 2>(c, j + 2, q);
        pre(j + 3); stage_plane<R, CV, NT, NS, 3>(c, j + 3, q);
        pre(j + 4); stage_plane<R, CV, NT, NS, 4>(c, j + 4, q);
        pre(j + 5); stage_plane<R, CV, NT, NS, 5>(c, j + 5, q);
        pre(j + 6); stage_plane<R, CV, NT, NS, 6>(c, j + 6, q);
        pre(j + 7); stage_plane<R, CV, NT, NS, 7>(c, j + 7, q);
        pre(j + 8); stage_plane<R, CV, NT, NS, 8>(c, j + 8, q);
    }
#pragma unroll 1
    for (; j < np; j++) {
        pre(j);
        switch (j % 9) {
        case 0: stage_plane<R, CV, NT, NS, 0>(c, j, q); break;
        case 1: stage_plane<R, CV, NT, NS, 1>(c, j, q); break;
        case 2: stage_plane<R, CV, NT, NS, 2>(c, j, q); break;
        case 3: stage_plane<R, CV, NT, NS, 3>(c, j, q); break;
        case 4: stage_plane<R, CV, NT, NS, 4>(c, j, q); break;
        case 5: stage_plane<R, CV, NT, NS, 5>(c, j, q); break;
        case 6: stage_plane<R, CV, NT, NS, 6>(c, j, q); break;
        case 7: stage_plane<R, CV, NT, NS, 7>(c, j, q); break;
        default: stage_plane<R, CV, NT, NS, 8>(c, j, q); break;
        }
    }
    cp_async_wait<0>();
}

// The staged kernel keeps its row table in dynamic shared memory after the
// pipeline slots, sized by the z-segment length (srow_off bytes in), so that
// MINB blocks fit on one SM.
template <typename R, int CV, int NS, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_apply_staged(const ApplyArgs<R> a, int nchunks, int srow_off) {
    extern __shared__ __align__(128) unsigned char smraw[];
    staged_block<R, CV, NS, NT>(a, a.tiles[blockIdx.x / nchunks], blockIdx.x % nchunks, smraw,
                                (SRow *)(smraw + srow_off));
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
    const int n = (rc.xmax - rc.xmin + 1) * SV;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int xo = t / SV, v = t - xo * SV;
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

// One thread per (point, vector) with the antisymmetric-image boundary of a
// box mesh (rsg_odd.cuh): every neighbour goes through the image rule; the
// diagonal, projectors and epilogue are those of the other kernels.
template <typename R>
__global__ void __launch_bounds__(256) k_apply_naive_odd(const ApplyArgs<R> a) {
    using V = VT<R>;
    using T = typename V::T;
    const int row = blockIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz, SV = a.SV;
    const int y = row % ny, z = row / ny;
    const Row rc = a.rows[row];
    if (rc.xmin > rc.xmax) return;
    const T *__restrict__ in = (const T *)a.in;
    const int n = (rc.xmax - rc.xmin + 1) * SV;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int xo = t / SV, v = t - xo * SV;
        const int x = rc.xmin + xo;
        const int64_t idx = (int64_t)rc.start + xo;
        const T c = V::ldg(in + idx * SV + v);
        T acc = V::scale((R)3 * a.w[0], c);
        for (int k = 1; k <= 4; k++) {
            T s = V::add(odd_site<R>(in, a.rows, x - k, y, z, nx, ny, nz, SV, v),
                         odd_site<R>(in, a.rows, x + k, y, z, nx, ny, nz, SV, v));
            s = V::add(s, odd_site<R>(in, a.rows, x, y - k, z, nx, ny, nz, SV, v));
            s = V::add(s, odd_site<R>(in, a.rows, x, y + k, z, nx, ny, nz, SV, v));
            s = V::add(s, odd_site<R>(in, a.rows, x, y, z - k, nx, ny, nz, SV, v));
            s = V::add(s, odd_site<R>(in, a.rows, x, y, z + k, nx, ny, nz, SV, v));
            V::fma(acc, a.w[k], s);
        }
        finish_point<R>(a, idx, x, y, z, v, c, acc);
    }
}

template <typename R>
cudaError_t launch_apply_naive_odd(const ApplyArgs<R> &a, cudaStream_t st) {
    if (a.ny * a.nz == 0) return cudaSuccess;
    k_apply_naive_odd<R><<<a.ny * a.nz, 256, 0, st>>>(a);
    return cudaGetLastError();
}

static inline int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

#if !defined(RSG_ONLY_DOUBLE) && !defined(RSG_ROWTMA_TU)
// Block shape of the staged kernel for SV vectors per point (shared with the
// host's tile builder through stage_shape()).
void stage_shape(const TileCfg &c, int SV, int *cv, int *nxr, int *ty) {
    int v = 1;
    while (v < SV && v < c.cv) v <<= 1;
    // 512 threads, or 256 for any other setting (192 is a kernel-5 shape)
    const int nt = c.threads == 512 ? 512 : 256;
    if (nt == 256 && v < 2) v = 2;
    if (nt == 256 && v > 4) v = 4;
    *cv = v;
    *ty = 16;          // fixed geometry: threads = cv x (threads / 16 / cv) x 16
    *nxr = nt / 16 / v;
}

size_t stage_smem_bytes(const TileCfg &c, int SV, size_t vec_bytes) {
    int cv, nxr, ty;
    stage_shape(c, SV, &cv, &nxr, &ty);
    // NS slots of the (ty + 8) x (nxr + 8) halo tile, plus per-thread base and V;
    // NS as launch_staged_cv picks it: 3 only with 256 threads and stages = 3
    // (the 512-thread instantiations always have 4)
    const int ns = (c.threads != 512 && c.stages == 3) ? 3 : 4;
    return (size_t)ns *
           ((size_t)(ty + 8) * (nxr + 8) * cv * vec_bytes + (size_t)cv * nxr * ty * (vec_bytes + vec_bytes / 2));
}

// Row-table bytes of the staged kernel: (ty + 8) rows x (zseg + 8) planes.
size_t stage_rows_bytes(const TileCfg &c) { return (size_t)(16 + 8) * (c.zseg + 8) * sizeof(SRow); }

// Block shape of the TMA kernel: 512 threads, one point per thread along x,
// pipeline (4 slots of the halo tile plus the base tile) within 200 KB.
void tma_shape(const TileCfg &c, int SV, int *cv, int *nxr, int *ty) {
    int v = 1;
    while (v < SV && v < c.cv) v <<= 1;
    *cv = v;
    int t = c.ty;
    while (v * t > 256 && t > 1) t >>= 1;
    *ty = t;
    int n = 512 / (v * t);
    while (n > 4 && (size_t)4 * ((size_t)(t + 8) * (n + 8) * v + (size_t)t * n * v) * 16 > 200 * 1024) n >>= 1;
    *nxr = n;
}
#else
size_t stage_smem_bytes(const TileCfg &c, int SV, size_t vec_bytes);
size_t stage_rows_bytes(const TileCfg &c);
#endif

template <typename R, int CV, int NS, int NT, int MINB>
static cudaError_t launch_staged_t(const ApplyArgs<R> &a, unsigned nblk, size_t smem, int srow_off,
                                   int nchunks, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_staged<R, CV, NS, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    using G = StagedGeom<CV, NT>;
    k_apply_staged<R, CV, NS, NT, MINB><<<nblk, dim3(CV, G::TX, G::TY), smem, st>>>(a, nchunks, srow_off);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_staged_cv(const ApplyArgs<R> &a, const TileCfg &cfg, int cv, unsigned nblk, size_t smem,
                                    int srow_off, int nchunks, cudaStream_t st) {
    if (cfg.threads != 512) {
        const bool three = cfg.blocks_per_sm >= 3;
        if (cfg.stages == 3) {
            if (cv <= 2)
                return three ? launch_staged_t<R, 2, 3, 256, 3>(a, nblk, smem, srow_off, nchunks, st)
                             : launch_staged_t<R, 2, 3, 256, 2>(a, nblk, smem, srow_off, nchunks, st);
            return three ? launch_staged_t<R, 4, 3, 256, 3>(a, nblk, smem, srow_off, nchunks, st)
                         : launch_staged_t<R, 4, 3, 256, 2>(a, nblk, smem, srow_off, nchunks, st);
        }
        if (cv <= 2)
            return three ? launch_staged_t<R, 2, 4, 256, 3>(a, nblk, smem, srow_off, nchunks, st)
                         : launch_staged_t<R, 2, 4, 256, 2>(a, nblk, smem, srow_off, nchunks, st);
        return three ? launch_staged_t<R, 4, 4, 256, 3>(a, nblk, smem, srow_off, nchunks, st)
                     : launch_staged_t<R, 4, 4, 256, 2>(a, nblk, smem, srow_off, nchunks, st);
    }
    switch (cv) {
    case 1: return launch_staged_t<R, 1, 4, 512, 1>(a, nblk, smem, srow_off, nchunks, st);
    case 2: return launch_staged_t<R, 2, 4, 512, 1>(a, nblk, smem, srow_off, nchunks, st);
    case 4: return launch_staged_t<R, 4, 4, 512, 1>(a, nblk, smem, srow_off, nchunks, st);
    default: return launch_staged_t<R, 8, 4, 512, 1>(a, nblk, smem, srow_off, nchunks, st);
    }
}

template <typename R>
cudaError_t launch_apply(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st) {
    if (cfg.kernel == 1) {
        k_apply_naive<R><<<a.ny * a.nz, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (ntiles == 0) return cudaSuccess;
    if (cfg.kernel == 2) {
        const int cv = pow2_at_least(a.SV) < 8 ? pow2_at_least(a.SV) : 8;
        int ty = cfg.ty;
        while (cv * ty > 256) ty >>= 1;
        const int nxr = 256 / (cv * ty);
        dim3 block(cv, nxr, ty);
        dim3 grid(ntiles, (a.SV + cv - 1) / cv);
        switch (cfg.rx) {
        case 1: k_apply_zmarch<R, 1><<<grid, block, 0, st>>>(a); break;
        case 2: k_apply_zmarch<R, 2><<<grid, block, 0, st>>>(a); break;
        default: k_apply_zmarch<R, 4><<<grid, block, 0, st>>>(a); break;
        }
        return cudaGetLastError();
    }
    int cv, nxr, ty;
    stage_shape(cfg, a.SV, &cv, &nxr, &ty);
    const int nchunks = (a.SV + cv - 1) / cv;
    const size_t slots = stage_smem_bytes(cfg, a.SV, sizeof(typename VT<R>::T));
    const size_t smem = slots + stage_rows_bytes(cfg);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const long long nblk = (long long)ntiles * nchunks;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if ((long long)a.P * a.SV >= 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_staged_cv<R>(a, cfg, cv, (unsigned)nblk, smem, (int)slots, nchunks, st);
}

// ---------------------------------------------------------- projectors ---
// Block: (BV vectors) x (PL point lanes).  Chunk c covers entries [q0, q1)
// of one atom.  partial[((c * npmax + i) * SV + v) * 2 * NC + comp] (FP64).
//
// With counter != nullptr the coefficients are finished in the same launch:
// after writing its partial sums a block counts itself done for its atom
// (per vector slice blockIdx.y), and the last block of an atom sums the
// atom's chunks in chunk order, scales by h^3 and applies h_a, exactly as
// k_proj_reduce does, then resets the counter for the next launch.
template <typename R, int NP>
__global__ void __launch_bounds__(256) k_proj_dot(const typename VT<R>::T *__restrict__ u, int SV,
                                                  const int32_t *__restrict__ q_pt,
                                                  const R *__restrict__ q_p,
                                                  const int32_t *__restrict__ chunk_q0,
                                                  const int32_t *__restrict__ chunk_q1,
                                                  double *__restrict__ partial,
                                                  unsigned *__restrict__ counter,
                                                  const int32_t *__restrict__ chunk_atom,
                                                  const int32_t *__restrict__ atom_chunk0,
                                                  const double *__restrict__ hm, double h3, R *__restrict__ D) {
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
        // UNR entries per iteration: their point indices, then their values,
        // are independent loads in flight together
        constexpr int UNR = 4;
        const int by = blockDim.y;
        int q = q0 + threadIdx.y;
        for (; q + (UNR - 1) * by < q1; q += UNR * by) {
            int pt[UNR];
#pragma unroll
            for (int k = 0; k < UNR; k++) pt[k] = q_pt[q + k * by];
            T val[UNR];
#pragma unroll
            for (int k = 0; k < UNR; k++) val[k] = V::ldg(u + (int64_t)pt[k] * SV + v);
#pragma unroll
            for (int k = 0; k < UNR; k++)
#pragma unroll
                for (int i = 0; i < NP; i++) V::fma(acc[i], q_p[(int64_t)(q + k * by) * NP + i], val[k]);
        }
        for (; q < q1; q += by) {
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
    if (counter == nullptr) return;
    // the last block of this atom and vector slice finishes its coefficients
    __shared__ int last;
    __threadfence();
    __syncthreads();
    const int at = chunk_atom[c];
    if (tid == 0) {
        const unsigned n = (unsigned)(atom_chunk0[at + 1] - atom_chunk0[at]);
        unsigned *cnt = counter + (size_t)at * gridDim.y + blockIdx.y;
        last = atomicAdd(cnt, 1u) == n - 1;
        if (last) *cnt = 0u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int ldc = SV * V::NC;
    const int s0 = blockIdx.y * blockDim.x * V::NC;                 // first complex column of the slice
    const int ns = min((int)blockDim.x * V::NC, ldc - s0);          // complex columns in the slice
    __shared__ double cbuf[2 * NP * 32 * V::NC];                    // c[i][s] of the slice (re, im)
    for (int t = tid; t < NP * ns; t += blockDim.x * blockDim.y) {
        const int i = t / ns, sc = s0 + (t - i * ns);
        double sr = 0.0, si = 0.0;
        for (int cc = atom_chunk0[at]; cc < atom_chunk0[at + 1]; cc++) {
            const double *pp = partial + (((int64_t)cc * NP + i) * ldc + sc) * 2;
            sr += __ldcg(pp);
            si += __ldcg(pp + 1);
        }
        cbuf[2 * t] = h3 * sr;
        cbuf[2 * t + 1] = h3 * si;
    }
    __syncthreads();
    for (int t = tid; t < NP * ns; t += blockDim.x * blockDim.y) {
        const int i = t / ns, sl = t - i * ns;
        double dr = 0.0, di = 0.0;
        for (int j = 0; j < NP; j++) {
            const double hij = hm[((int64_t)at * NP + i) * NP + j];
            dr += hij * cbuf[2 * (j * ns + sl)];
            di += hij * cbuf[2 * (j * ns + sl) + 1];
        }
        R *dst = D + (((int64_t)at * NP + i) * ldc + s0 + sl) * 2;
        dst[0] = (R)dr;
        dst[1] = (R)di;
    }
}

template <typename R>
cudaError_t launch_proj_dot(const void *u, int SV, const ProjDev &pj, double *partial,
                            cudaStream_t st) {
    return launch_proj_coeffs<R>(u, SV, pj, partial, nullptr, 0.0, nullptr, st);
}

template <typename R>
cudaError_t launch_proj_coeffs(const void *u, int SV, const ProjDev &pj, double *partial, unsigned *counter,
                               double h3, void *D, cudaStream_t st) {
    if (pj.natoms == 0 || pj.nchunks == 0) return cudaSuccess;
    const int bv = SV < 32 ? SV : 32;
    const int pl = 256 / bv > 64 ? 64 : 256 / bv;
    dim3 block(bv, pl);
    dim3 grid(pj.nchunks, proj_slices(SV));
    using T = typename VT<R>::T;
    const T *uu = (const T *)u;
    const R *qp = (const R *)pj.q_p;
    R *DD = (R *)D;
#define RSG_PROJ_DOT(NP_)                                                                                     \
    k_proj_dot<R, NP_><<<grid, block, 0, st>>>(uu, SV, pj.q_pt, qp, pj.chunk_q0, pj.chunk_q1, partial, counter, \
                                               pj.chunk_atom, pj.atom_chunk0, pj.hm, h3, DD)
    switch (pj.npmax) {
    case 1: RSG_PROJ_DOT(1); break;
    case 4: RSG_PROJ_DOT(4); break;
    case 9: RSG_PROJ_DOT(9); break;
    default: return cudaErrorInvalidValue;
    }
#undef RSG_PROJ_DOT
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
#pragma unroll 4
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

// Projector terms of H u added to an already written result:
//     out[p, v] += alpha * sum_{entries (a, q) at p} sum_i p_ai(q) D[a, i, v]
//     acc[p, v] += gamma * alpha * (same)            (when acc is used)
// one thread per (union point, vector); the union points and their entry
// lists come from the point-centric CSR, so there are no atomics.
// Each block row (threadIdx.y) takes kScatPts union points, blockDim.y rows
// apart; their index, state and first-entry loads are issued before any of
// them is used, so that several points' loads are in flight per warp.
constexpr int kScatPts = 4;
template <typename R>
__global__ void __launch_bounds__(256) k_proj_scatter(const ApplyArgs<R> a, const int32_t *__restrict__ upts,
                                                      const int32_t *__restrict__ uptr,
                                                      const int32_t *__restrict__ e_atom,
                                                      const R *__restrict__ e_p, int nu) {
    using V = VT<R>;
    using T = typename V::T;
    const int ub = blockIdx.x * blockDim.y * kScatPts + threadIdx.y;
    const T *D = (const T *)a.D;
    T *out = (T *)a.out;
    int p[kScatPts], e0[kScatPts], e1[kScatPts], at0[kScatPts];
#pragma unroll
    for (int k = 0; k < kScatPts; k++) {
        const int u = ub + k * (int)blockDim.y;
        const bool ok = u < nu;
        p[k] = ok ? upts[u] : -1;
        e0[k] = ok ? uptr[u] : 0;
        e1[k] = ok ? uptr[u + 1] : 0;
    }
#pragma unroll
    for (int k = 0; k < kScatPts; k++) at0[k] = e1[k] > e0[k] ? e_atom[e0[k]] : 0;
    for (int v = threadIdx.x; v < a.SV; v += blockDim.x) {
        T o[kScatPts];
#pragma unroll
        for (int k = 0; k < kScatPts; k++) o[k] = p[k] >= 0 ? out[(int64_t)p[k] * a.SV + v] : V::zero();
#pragma unroll
        for (int k = 0; k < kScatPts; k++) {
            if (p[k] < 0) continue;
            T sum = V::zero();
            for (int e = e0[k]; e < e1[k]; e++) {
                const int at = e == e0[k] ? at0[k] : e_atom[e];
                const R *pv = e_p + (int64_t)e * a.npmax;
                const T *Da = D + (int64_t)at * a.npmax * a.SV + v;
                for (int i = 0; i < a.npmax; i++) V::fma(sum, pv[i], Da[(int64_t)i * a.SV]);
            }
            const int64_t oi = (int64_t)p[k] * a.SV + v;
            const T y = V::cmul(a.ar, a.ai, sum);
            out[oi] = V::add(o[k], y);
            if (a.acc != nullptr) {
                T sacc = ((T *)a.acc)[oi];
                V::cfma(sacc, a.gr, a.gi, y);
                ((T *)a.acc)[oi] = sacc;
            }
        }
    }
}

template <typename R>
cudaError_t launch_proj_scatter(const ApplyArgs<R> &a, const ProjDev &pj, cudaStream_t st) {
    const int nu = pj.nu;
    if (nu == 0) return cudaSuccess;
    const int bx = a.SV < 32 ? a.SV : 32;
    const int by = 256 / bx;
    const int per = by * kScatPts;
    k_proj_scatter<R><<<(nu + per - 1) / per, dim3(bx, by), 0, st>>>(a, pj.u_pts, pj.u_ptr, pj.e_atom,
                                                                    (const R *)pj.e_p, nu);
    return cudaGetLastError();
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

// ----------------------------------------------------------- TMA gather ---
// k_apply_tma: the staged z-march with the plane tiles brought in by the
// tensor memory accelerator.  Warp 0 gathers each plane's (TY+8) x (TX+8)
// points, four arbitrary point indices per cp.async.bulk.tensor...gather4
// (points outside the mesh get the out-of-range index P, which the TMA
// zero-fills), plus the base values of the outputs retired at that plane;
// completion is tracked by one mbarrier per slot.  The other warps only
// compute.  Every mbarrier wait is bounded: on timeout the block records an
// error (a.err = 2) and leaves at the next block barrier.
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_arrive(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_gather4(unsigned dst, const CUtensorMap *tm, int col, int r0, int r1,
                                            int r2, int r3, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(tm), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
}

constexpr long kWaitLimit = 1L << 22;   // try_wait polls before a slot is declared lost

template <typename R, int CV, int NS>
__global__ void __launch_bounds__(512, 1) k_apply_tma(const ApplyArgs<R> a, const __grid_constant__ CUtensorMap tm_in,
                                                      const __grid_constant__ CUtensorMap tm_base, int nchunks,
                                                      int *err) {
    using V = VT<R>;
    using T = typename V::T;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ SRow srows[kSRows];
    __shared__ __align__(8) unsigned long long mbar[NS];
    const int NXR = blockDim.y, TY = blockDim.z;
    const int TX = NXR, WX = TX + 8, WY = TY + 8;
    const int chunk = blockIdx.x % nchunks;
    const Tile tl = a.tiles[blockIdx.x / nchunks];
    const int ny = a.ny, nz = a.nz, SV = a.SV, P = (int)a.P;
    const int xbase = tl.tx * TX - 4, ybase = tl.ty * TY - 4, zbase = tl.zlo - 4;
    const int nzr = tl.zhi - tl.zlo + 8;
    const int nthr = CV * NXR * TY;
    const int tid = (threadIdx.z * NXR + threadIdx.y) * CV + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < WY * nzr; i += nthr) {
        const int zz = i / WY;
        const int yy = ybase + (i - zz * WY);
        const int zg = zbase + zz;
        SRow r{0, 1, 0};
        if (yy >= 0 && yy < ny && zg >= 0 && zg < nz) {
            const Row g = a.rows[zg * ny + yy];
            r.start = g.start;
            r.xmin = (int16_t)g.xmin;
            r.xmax = (int16_t)g.xmax;
        }
        srows[i] = r;
    }
    const unsigned mbar0 = (unsigned)__cvta_generic_to_shared(mbar);
    if (tid == 0) {
        for (int k = 0; k < NS; k++) mbar_init(mbar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int slot_elems = WY * WX * CV, bslot_elems = TY * TX * CV;
    // tensor copies need 128-byte aligned destinations: round the dynamic
    // region up (the launch reserves 128 bytes of slack); with TX % 4 == 0
    // and CV >= 2 every slot and every four-point group is then aligned
    const unsigned raw = (unsigned)__cvta_generic_to_shared(smraw);
    T *slots = (T *)(smraw + ((128u - (raw & 127u)) & 127u));
    T *bslots = slots + NS * slot_elems;
    const unsigned sh_slots = (unsigned)__cvta_generic_to_shared(slots);
    const unsigned sh_bslots = (unsigned)__cvta_generic_to_shared(bslots);
    const int col = chunk * CV * (int)(16 / sizeof(R));     // element column of this chunk
    const bool has_base = a.base != nullptr;
    const unsigned tx_bytes = (unsigned)(slot_elems + (has_base ? bslot_elems : 0)) * 16u;
    const unsigned tx_bytes_nobase = (unsigned)slot_elems * 16u;

    // warp 0: gather plane j and the base of outputs retired at plane j
    auto issue = [&](int j) {
        const int sl = j % NS;
        const unsigned bar = mbar0 + 8 * sl;
        const SRow *rr = srows + j * WY;
        for (int g = lane; g < WY * WX / 4; g += 32) {
            int idx[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int pi = 4 * g + t;
                const int yy = pi / WX, xx = pi - yy * WX;
                const SRow rw = rr[yy];
                const int x = xbase + xx;
                idx[t] = (x >= rw.xmin && x <= rw.xmax) ? rw.start + (x - rw.xmin) : P;
            }
            const unsigned dst = sh_slots + (unsigned)((sl * slot_elems + 4 * g * CV) * 16);
            if (dst & 127u) {   // never expected: record it and leave the slot incomplete
                atomicExch(err, 3);
                continue;
            }
            tma_gather4(dst, &tm_in, col, idx[0], idx[1], idx[2], idx[3], bar);
        }
        const bool base_now = has_base && j >= 4;
        if (base_now) {
            const SRow *ro = srows + (j - 4) * WY + 4;
            for (int g = lane; g < TY * TX / 4; g += 32) {
                int idx[4];
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const int pi = 4 * g + t;
                    const int yi = pi / TX, xi = pi - yi * TX;
                    const SRow rw = ro[yi];
                    const int x = tl.tx * TX + xi;
                    idx[t] = (x >= rw.xmin && x <= rw.xmax) ? rw.start + (x - rw.xmin) : P;
                }
                const unsigned dst = sh_bslots + (unsigned)((sl * bslot_elems + 4 * g * CV) * 16);
                if (dst & 127u) {
                    atomicExch(err, 3);
                    continue;
                }
                tma_gather4(dst, &tm_base, col, idx[0], idx[1], idx[2], idx[3], bar);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_expect_arrive(bar, base_now ? tx_bytes : tx_bytes_nobase);
    };

    const int cv = threadIdx.x, xr = threadIdx.y, yi = threadIdx.z;
    const int v = chunk * CV + cv;
    const int y = tl.ty * TY + yi;
    const int x = tl.tx * TX + xr;
    const R w1 = a.w[1], w2 = a.w[2], w3 = a.w[3], w4 = a.w[4], w03 = (R)3 * a.w[0];
    // own potential, two planes ahead in registers
    auto vload = [&](int j) -> R {
        if (j >= nzr) return (R)0;
        const SRow rw = srows[j * WY + yi + 4];
        return (x >= rw.xmin && x <= rw.xmax) ? a.V[rw.start + (x - rw.xmin)] : (R)0;
    };
    R vq0 = vload(0), vq1 = vload(1);
    T q[9];
#pragma unroll
    for (int k = 0; k < 9; k++) q[k] = V::zero();
    if (warp == 0)
        for (int j = 0; j < NS - 1 && j < nzr; j++) issue(j);
    const int rs = WX * CV;
    int abort = 0;
    for (int j = 0; j < nzr; j++) {
        if (warp == 0 && j + NS - 1 < nzr) issue(j + NS - 1);
        const R vq2 = vload(j + 2);
        const unsigned bar = mbar0 + 8 * (j % NS);
        bool ok = false;
        for (long it = 0; it < kWaitLimit; ++it)
            if (mbar_try(bar, (unsigned)((j / NS) & 1))) {
                ok = true;
                break;
            }
        if (!ok) abort = 1;
        if (ok) {
            const T *sl = slots + (j % NS) * slot_elems;
            const T *cp = sl + ((yi + 4) * WX + xr + 4) * CV + cv;
            const T cval = cp[0];
            const int p = zbase + j;
            // queue rotates by renaming inside the nine-way unrolled body below
            T s = V::scale(w03, cval);
            V::fma(s, w1, V::add(V::add(cp[-CV], cp[CV]), V::add(cp[-rs], cp[rs])));
            V::fma(s, w2, V::add(V::add(cp[-2 * CV], cp[2 * CV]), V::add(cp[-2 * rs], cp[2 * rs])));
            V::fma(s, w3, V::add(V::add(cp[-3 * CV], cp[3 * CV]), V::add(cp[-3 * rs], cp[3 * rs])));
            V::fma(s, w4, V::add(V::add(cp[-4 * CV], cp[4 * CV]), V::add(cp[-4 * rs], cp[4 * rs])));
            const R diag = vq0 + a.f0 + a.fx * (R)x + a.fy * (R)y + a.fz * (R)p;
            V::fma(s, diag, cval);
            // shift-free queue: output p+k-4 lives in q[(k + j) % 9]
            const int jm = j % 9;
            switch (jm) {
#define RSG_PHASE(PH)                                                                          \
    case PH: {                                                                                 \
        constexpr int Q0 = (0 + PH) % 9, Q1 = (1 + PH) % 9, Q2 = (2 + PH) % 9, Q3 = (3 + PH) % 9; \
        constexpr int Q4 = (4 + PH) % 9, Q5 = (5 + PH) % 9, Q6 = (6 + PH) % 9, Q7 = (7 + PH) % 9; \
        constexpr int Q8 = (8 + PH) % 9;                                                       \
        V::fma(q[Q3], w1, cval);                                                               \
        V::fma(q[Q5], w1, cval);                                                               \
        V::fma(q[Q2], w2, cval);                                                               \
        V::fma(q[Q6], w2, cval);                                                               \
        V::fma(q[Q1], w3, cval);                                                               \
        V::fma(q[Q7], w3, cval);                                                               \
        V::fma(q[Q0], w4, cval);                                                               \
        V::fma(q[Q8], w4, cval);                                                               \
        q[Q4] = V::add(q[Q4], s);                                                              \
        if (p - 4 >= tl.zlo && p - 4 < tl.zhi && v < SV) {                                     \
            const SRow ro = srows[(j - 4) * WY + yi + 4];                                      \
            if (x >= ro.xmin && x <= ro.xmax) {                                                \
                const int o = (ro.start + (x - ro.xmin)) * SV + v;                             \
                const T bv = bslots[((j % NS) * TY + yi) * TX * CV + xr * CV + cv];            \
                finish_staged<R>(a, o, q[Q0], bv);                                             \
            }                                                                                  \
        }                                                                                      \
        q[Q0] = V::zero();                                                                     \
    } break;
                RSG_PHASE(0)
                RSG_PHASE(1)
                RSG_PHASE(2)
                RSG_PHASE(3)
                RSG_PHASE(4)
                RSG_PHASE(5)
                RSG_PHASE(6)
                RSG_PHASE(7)
                RSG_PHASE(8)
#undef RSG_PHASE
            }
        }
        vq0 = vq1;
        vq1 = vq2;
        // barrier-OR: every thread takes the same decision
        if (__syncthreads_or(abort)) {
            if (tid == 0) {
                atomicExch(err, 2);
                // leave only after the copies still in flight (planes up to
                // j + NS - 1, one per slot) have landed, each wait bounded
                const int last = min(nzr - 1, j + NS - 1);
                for (int jp = max(0, last - NS + 1); jp <= last; jp++) {
                    const unsigned b = mbar0 + 8 * (jp % NS), par = (unsigned)((jp / NS) & 1);
                    for (long it = 0; it < kWaitLimit; ++it)
                        if (mbar_try(b, par)) break;
                }
            }
            __syncthreads();
            return;
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D view of a (P, SV) block of 16-byte vectors as R elements: rows are
// points, a box is one point's CV vectors.
template <typename R>
static bool encode_rows(CUtensorMap *tm, const void *base, int64_t P, int SV, int CV) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !base) return false;
    const int epv = 16 / (int)sizeof(R);
    cuuint64_t dims[2] = {(cuuint64_t)SV * epv, (cuuint64_t)P};
    cuuint64_t strides[1] = {(cuuint64_t)SV * 16};
    cuuint32_t box[2] = {(cuuint32_t)(CV * epv), 1};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt = sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return fn(tm, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename R, int CV>
static cudaError_t launch_tma_cv(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, int nxr, int ty,
                                 cudaStream_t st, bool *launched) {
    constexpr int NS = 4;
    CUtensorMap tm_in, tm_base;
    if (!encode_rows<R>(&tm_in, a.in, a.P, a.SV, CV)) return cudaSuccess;
    if (!encode_rows<R>(&tm_base, a.base ? a.base : a.in, a.P, a.SV, CV)) return cudaSuccess;
    const int WX = nxr + 8, WY = ty + 8;
    const size_t smem = (size_t)NS * ((size_t)WY * WX * CV + (size_t)ty * nxr * CV) * 16 + 128;
    cudaError_t e = cudaFuncSetAttribute(k_apply_tma<R, CV, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nchunks = (a.SV + CV - 1) / CV;
    k_apply_tma<R, CV, NS><<<(unsigned)((long long)ntiles * nchunks), dim3(CV, nxr, ty), smem, st>>>(
        a, tm_in, tm_base, nchunks, a.err);
    *launched = true;
    (void)cfg;
    return cudaGetLastError();
}

// Returns with *launched = false when the TMA path does not apply (no
// encoder, tile width not a multiple of 4, too much shared memory).
template <typename R>
cudaError_t launch_apply_tma(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                             bool *launched) {
    *launched = false;
    if (ntiles == 0 || a.err == nullptr || (long long)a.P >= 0x7fffffffLL) return cudaSuccess;
    int cv, nxr, ty;
    tma_shape(cfg, a.SV, &cv, &nxr, &ty);
    // four-point groups of at least 128 bytes keep every destination aligned
    if (nxr % 4 != 0 || cv < 2) return cudaSuccess;
    switch (cv) {
    case 2: return launch_tma_cv<R, 2>(a, cfg, ntiles, nxr, ty, st, launched);
    case 4: return launch_tma_cv<R, 4>(a, cfg, ntiles, nxr, ty, st, launched);
    default: return launch_tma_cv<R, 8>(a, cfg, ntiles, nxr, ty, st, launched);
    }
}

// ------------------------------------------------------ row-TMA staged ---
// k_apply_rowtma: the z-march of k_apply_staged with every state plane
// brought in by the tensor memory accelerator one mesh row at a time.  In
// the row-contiguous point order a tile's row segment (WX points in the TY
// middle rows, the TX interior points in the four halo rows above and below)
// is a run of consecutive point indices, so one tiled copy of a (CV vectors)
// x (segment) box over the 2-D view (points, state columns) fetches it.
// Where a segment runs past an end of its mesh row the copy brings points of
// the neighbouring rows (or the zero fill beyond the array); warp 1 zeroes
// those entries one plane ahead, after the copy has landed and before the
// block barrier that precedes their first read.  Segments that miss their
// row are not copied and are zeroed whole.  Warp 0 issues the copies (one
// lane per row) and arms the slot's mbarrier with the byte count; all warps
// compute.  Per thread and plane the only other memory work is the potential
// of its point two planes ahead (registers) and one cp.async of the base
// value of an output retired NS - 1 planes later.  Each thread keeps the
// point indices of its column in a ring of eight planes in shared memory.
// Every mbarrier wait is bounded; a wait that gives up makes the whole block
// leave at the next barrier (a barrier-OR, so the decision is uniform) after
// a bounded wait for its copies in flight, with err = 2.
template <int CV, int NS, int NT>
struct RowTmaSmem {
    using G = StagedGeom<CV, NT>;
    static constexpr size_t SLOTS = (size_t)NS * G::SLOT * 16;    // state planes
    static constexpr size_t BSLOTS = (size_t)NS * NT * 16;        // base values
    static constexpr size_t IDX = (size_t)8 * NT * 4;              // point-index ring
    static constexpr size_t ROWS_OFF = SLOTS + BSLOTS + IDX;
    // 128 bytes of slack: the region is rounded up to a 128-byte boundary
    static size_t bytes(int zseg) { return 128 + ROWS_OFF + (size_t)G::WY * (zseg + 8) * sizeof(SRow); }
};

__device__ __forceinline__ void tma_tile2d(unsigned dst, const CUtensorMap *tm, int c0, int c1, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tm), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

template <typename R, int CV, int NT>
struct RtCtx {
    using T = typename VT<R>::T;
    const T *slots;
    const T *bslots;
    const int *idxr;
    int tid, xr, yi, cv, v;
    bool vok;
    int zbase;
    R fxy;                       // f0 + fx x + fy y of the thread's column
    R w0, w1, w2, w3, w4;
};

// Plane j has landed (and been fixed up): add its contributions, retire
// output j - 4.  Queue slot of output j + (k - 4) is (k + PH) % 9.
template <typename R, int CV, int NT, int NS, int PH>
__device__ __forceinline__ void rt_plane(const ApplyArgs<R> &a, const RtCtx<R, CV, NT> &c, int j, bool on,
                                         R vj, typename VT<R>::T (&q)[9]) {
    using V = VT<R>;
    using T = typename V::T;
    using G = StagedGeom<CV, NT>;
    constexpr int Q0 = (0 + PH) % 9, Q1 = (1 + PH) % 9, Q2 = (2 + PH) % 9, Q3 = (3 + PH) % 9;
    constexpr int Q4 = (4 + PH) % 9, Q5 = (5 + PH) % 9, Q6 = (6 + PH) % 9, Q7 = (7 + PH) % 9;
    constexpr int Q8 = (8 + PH) % 9;
    constexpr int RS = G::WX * CV;
    const T *sl = c.slots + (j % NS) * G::SLOT;
    const T *cp = sl + ((c.yi + 4) * G::WX + c.xr + 4) * CV + c.cv;
    if (on) {   // the thread's column has a mesh point at plane j
        const T cval = cp[0];
        V::fma(q[Q3], c.w1, cval);
        V::fma(q[Q5], c.w1, cval);
        V::fma(q[Q2], c.w2, cval);
        V::fma(q[Q6], c.w2, cval);
        V::fma(q[Q1], c.w3, cval);
        V::fma(q[Q7], c.w3, cval);
        V::fma(q[Q0], c.w4, cval);
        V::fma(q[Q8], c.w4, cval);
        T s = V::scale((R)3 * c.w0, cval);
        V::fma(s, c.w1, V::add(V::add(cp[-CV], cp[CV]), V::add(cp[-RS], cp[RS])));
        V::fma(s, c.w2, V::add(V::add(cp[-2 * CV], cp[2 * CV]), V::add(cp[-2 * RS], cp[2 * RS])));
        V::fma(s, c.w3, V::add(V::add(cp[-3 * CV], cp[3 * CV]), V::add(cp[-3 * RS], cp[3 * RS])));
        V::fma(s, c.w4, V::add(V::add(cp[-4 * CV], cp[4 * CV]), V::add(cp[-4 * RS], cp[4 * RS])));
        const R diag = vj + c.fxy + a.fz * (R)(c.zbase + j);
        V::fma(s, diag, cval);
        q[Q4] = V::add(q[Q4], s);
    }
    // output plane j - 4 lies in [zlo, zhi) for j in [8, np)
    if (j >= 8 && c.vok) {
        const int id = c.idxr[((j - 4) & 7) * NT + c.tid];
        if (id >= 0) finish_staged<R>(a, id * a.SV + c.v, q[Q0], c.bslots[(j % NS) * NT + c.tid]);
    }
    q[Q0] = V::zero();
}

template <typename R, int CV, int NS, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_apply_rowtma(const ApplyArgs<R> a, const __grid_constant__ CUtensorMap tm_mid,
                   const __grid_constant__ CUtensorMap tm_halo, int nchunks) {
    using V = VT<R>;
    using T = typename V::T;
    using G = StagedGeom<CV, NT>;
    using L = RowTmaSmem<CV, NS, NT>;
    static_assert(CV % 2 == 0, "row copies need 128-byte aligned shared-memory rows");
    static_assert(NS >= 4 && NS <= 7, "base staging distance");
    constexpr int TX = G::TX, TY = G::TY, WX = G::WX, WY = G::WY;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long mbar[NS];
    const unsigned raw = (unsigned)__cvta_generic_to_shared(smraw);
    unsigned char *sm = smraw + ((128u - (raw & 127u)) & 127u);
    T *slots = (T *)sm;
    T *bslots = (T *)(sm + L::SLOTS);
    int *idxr = (int *)(sm + L::SLOTS + L::BSLOTS);
    SRow *srows = (SRow *)(sm + L::ROWS_OFF);

    const int chunk = blockIdx.x % nchunks;
    const Tile tl = a.tiles[blockIdx.x / nchunks];
    const int ny = a.ny, nz = a.nz, SV = a.SV;
    const int xbase = tl.tx * TX - 4, ybase = tl.ty * TY - 4, zbase = tl.zlo - 4;
    const int np = tl.zhi - tl.zlo + 8;
    const int tid = (threadIdx.z * TX + threadIdx.y) * CV + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < WY * np; i += NT) {
        const int zz = i / WY;
        const int yy = ybase + (i - zz * WY);
        const int zg = zbase + zz;
        SRow r{0, 1, 0};
        if (yy >= 0 && yy < ny && zg >= 0 && zg < nz) {
            const Row g = a.rows[zg * ny + yy];
            r.start = g.start;
            r.xmin = (int16_t)g.xmin;
            r.xmax = (int16_t)g.xmax;
        }
        srows[i] = r;
    }
    const unsigned mbar0 = (unsigned)__cvta_generic_to_shared(mbar);
    if (tid == 0) {
        for (int k = 0; k < NS; k++) mbar_init(mbar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const unsigned sh_slots = (unsigned)__cvta_generic_to_shared(slots);
    const int col = chunk * CV * (int)(16 / sizeof(R));     // element column of this chunk
    // row yy's segment: first x, width and offset in the slot (16-byte entries)
    auto seg = [&](int yy, int &xs, int &w, int &off) {
        const bool mid = yy >= 4 && yy < 4 + TY;
        xs = mid ? xbase : xbase + 4;
        w = mid ? WX : TX;
        off = (yy * WX + (mid ? 0 : 4)) * CV;
    };
    // warp 0: copy the row segments of plane jp, arm its mbarrier
    auto issue = [&](int jp) {
        const int sl = jp % NS;
        const unsigned bar = mbar0 + 8u * (unsigned)sl;
        bool go = false, mid = false;
        int pidx = 0, off = 0;
        if (lane < WY) {
            int xs, w;
            seg(lane, xs, w, off);
            mid = w == WX;
            const SRow rw = srows[jp * WY + lane];
            go = rw.xmin <= rw.xmax && xs <= rw.xmax && xs + w - 1 >= rw.xmin;
            pidx = rw.start + (xs - rw.xmin);
        }
        const unsigned bm = __ballot_sync(0xffffffffu, go && mid);
        const unsigned bh = __ballot_sync(0xffffffffu, go && !mid);
        if (lane == 0) mbar_expect_arrive(bar, (unsigned)((__popc(bm) * WX + __popc(bh) * TX) * CV * 16));
        if (go) tma_tile2d(sh_slots + (unsigned)((sl * G::SLOT + off) * 16), mid ? &tm_mid : &tm_halo, col, pidx, bar);
    };
    auto wait_plane = [&](int jp) -> bool {
        const unsigned bar = mbar0 + 8u * (unsigned)(jp % NS);
        const unsigned par = (unsigned)((jp / NS) & 1);
        for (long it = 0; it < kWaitLimit; ++it)
            if (mbar_try(bar, par)) return true;
        return false;
    };
    // warp 1: zero the entries of plane jf that are not mesh points of their row
    auto fix = [&](int jf) {
        T *sl = slots + (jf % NS) * G::SLOT;
        int nl = 0, nr = 0, w = 0, off = 0;
        if (lane < WY) {
            int xs;
            seg(lane, xs, w, off);
            const SRow rw = srows[jf * WY + lane];
            if (rw.xmin > rw.xmax || xs > rw.xmax || xs + w - 1 < rw.xmin) {
                nl = w;
            } else {
                nl = max(0, rw.xmin - xs);
                nr = max(0, xs + w - 1 - rw.xmax);
            }
        }
        unsigned need = __ballot_sync(0xffffffffu, (nl | nr) != 0);
        while (need) {
            const int r = __ffs(need) - 1;
            need &= need - 1;
            const int rl = __shfl_sync(0xffffffffu, nl, r), rr = __shfl_sync(0xffffffffu, nr, r);
            const int rw = __shfl_sync(0xffffffffu, w, r), ro = __shfl_sync(0xffffffffu, off, r);
            for (int e = lane; e < rw * CV; e += 32) {
                const int xx = e / CV;
                if (xx < rl || xx >= rw - rr) sl[ro + e] = V::zero();
            }
        }
        // order these generic-proxy writes before the slot's next tensor copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };

    RtCtx<R, CV, NT> c;
    c.slots = slots;
    c.bslots = bslots;
    c.idxr = idxr;
    c.tid = tid;
    c.xr = threadIdx.y;
    c.yi = threadIdx.z;
    c.cv = threadIdx.x;
    c.v = chunk * CV + threadIdx.x;
    c.vok = c.v < SV;
    c.zbase = zbase;
    const int x = tl.tx * TX + threadIdx.y, y = tl.ty * TY + threadIdx.z, yown = threadIdx.z + 4;
    c.fxy = a.f0 + a.fx * (R)x + a.fy * (R)y;
    c.w0 = a.w[0];
    c.w1 = a.w[1];
    c.w2 = a.w[2];
    c.w3 = a.w[3];
    c.w4 = a.w[4];
    int *my_idx = idxr + tid;
    auto idx_of = [&](int jp) -> int {
        if (jp >= np) return -1;
        const SRow rw = srows[jp * WY + yown];
        return (x >= rw.xmin && x <= rw.xmax) ? rw.start + (x - rw.xmin) : -1;
    };
    const unsigned sh_b = (unsigned)__cvta_generic_to_shared(bslots);
    const T *__restrict__ basep = (const T *)a.base;
    // base value of output plane o into the slot its retirement (plane o + 4) reads
    auto stage_base = [&](int o) {
        if (basep != nullptr && o >= 4 && o < np - 4) {
            const int id = my_idx[(o & 7) * NT];
            const bool ok = id >= 0 && c.vok;
            cp_async16(sh_b + (unsigned)((((o + 4) % NS) * NT + tid) * 16), basep + (ok ? id * SV + c.v : 0),
                       ok ? 16 : 0);
        }
    };

    T q[9];
#pragma unroll
    for (int k = 0; k < 9; k++) q[k] = V::zero();
    int abort = 0;
    {
        const int i0 = idx_of(0), i1 = idx_of(1);
        my_idx[0] = i0;
        my_idx[NT] = i1;
    }
    R vq0 = my_idx[0] >= 0 ? a.V[my_idx[0]] : (R)0;
    R vq1 = my_idx[NT] >= 0 ? a.V[my_idx[NT]] : (R)0;
    unsigned okq = (my_idx[0] >= 0 ? 1u : 0u) | (my_idx[NT] >= 0 ? 2u : 0u);
    if (warp == 0)
        for (int k = 0; k < NS - 1 && k < np; k++) issue(k);
    if (warp == 1) {
        if (wait_plane(0)) fix(0);
        else abort = 1;
    }
    // iteration j: the barrier publishes plane j (landed, fixed) and frees the
    // slot of plane j - 1 for plane j + NS - 1; warp 1 fixes plane j + 1
    int last_issued = min(np, NS - 1) - 1;
    auto pre = [&](int j, R &vq2) -> bool {
        cp_async_wait<NS - 2>();
        if (__syncthreads_or(abort)) return true;
        if (warp == 0 && j + NS - 1 < np) issue(j + NS - 1);
        last_issued = min(np - 1, j + NS - 1);
        if (warp == 1 && j + 1 < np) {
            if (wait_plane(j + 1)) fix(j + 1);
            else abort = 1;
        }
        const int i2 = idx_of(j + 2);
        my_idx[((j + 2) & 7) * NT] = i2;
        vq2 = i2 >= 0 ? a.V[i2] : (R)0;
        okq |= (i2 >= 0 ? 4u : 0u);
        stage_base(j + NS - 5);
        cp_async_commit();
        if (!wait_plane(j)) abort = 1;   // already complete: warp 1 saw it before the barrier
        return false;
    };
    auto post = [&](R vq2) {
        vq0 = vq1;
        vq1 = vq2;
        okq >>= 1;
    };
    int j = 0;
    bool stop = false;
#define RSG_RT_STEP(PH)                                              \
    {                                                                \
        R vq2;                                                       \
        if (pre(j + PH, vq2)) {                                      \
            stop = true;                                             \
            break;                                                   \
        }                                                            \
        rt_plane<R, CV, NT, NS, PH>(a, c, j + PH, okq & 1u, vq0, q); \
        post(vq2);                                                   \
    }
#pragma unroll 1
    for (; j + 9 <= np; j += 9) {
        RSG_RT_STEP(0)
        RSG_RT_STEP(1)
        RSG_RT_STEP(2)
        RSG_RT_STEP(3)
        RSG_RT_STEP(4)
        RSG_RT_STEP(5)
        RSG_RT_STEP(6)
        RSG_RT_STEP(7)
        RSG_RT_STEP(8)
    }
#undef RSG_RT_STEP
    if (!stop) {
#pragma unroll 1
        for (; j < np; j++) {
            R vq2;
            if (pre(j, vq2)) {
                stop = true;
                break;
            }
            const bool on = okq & 1u;
            switch (j % 9) {
            case 0: rt_plane<R, CV, NT, NS, 0>(a, c, j, on, vq0, q); break;
            case 1: rt_plane<R, CV, NT, NS, 1>(a, c, j, on, vq0, q); break;
            case 2: rt_plane<R, CV, NT, NS, 2>(a, c, j, on, vq0, q); break;
            case 3: rt_plane<R, CV, NT, NS, 3>(a, c, j, on, vq0, q); break;
            case 4: rt_plane<R, CV, NT, NS, 4>(a, c, j, on, vq0, q); break;
            case 5: rt_plane<R, CV, NT, NS, 5>(a, c, j, on, vq0, q); break;
            case 6: rt_plane<R, CV, NT, NS, 6>(a, c, j, on, vq0, q); break;
            case 7: rt_plane<R, CV, NT, NS, 7>(a, c, j, on, vq0, q); break;
            default: rt_plane<R, CV, NT, NS, 8>(a, c, j, on, vq0, q); break;
            }
            post(vq2);
        }
    }
    cp_async_wait<0>();
    if (stop) {
        // leave only after the copies still in flight have landed (bounded)
        if (tid == 0) {
            atomicExch(a.err, 2);
            for (int jp = max(0, last_issued - NS + 1); jp <= last_issued; jp++) wait_plane(jp);
        }
        __syncthreads();
    }
}

// 2-D view of a (P, SV) block of 16-byte vectors as R elements: rows are
// points; a box is CV vectors of `rows` consecutive points.
template <typename R>
static bool encode_row_box(CUtensorMap *tm, const void *base, int64_t P, int SV, int CV, int rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !base || rows < 1 || rows > 256) return false;
    const int epv = 16 / (int)sizeof(R);
    cuuint64_t dims[2] = {(cuuint64_t)SV * epv, (cuuint64_t)P};
    cuuint64_t strides[1] = {(cuuint64_t)SV * 16};
    cuuint32_t box[2] = {(cuuint32_t)(CV * epv), (cuuint32_t)rows};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt = sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return fn(tm, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename R, int CV, int NS, int NT, int MINB>
static cudaError_t launch_rowtma_t(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                                   bool *launched) {
    using G = StagedGeom<CV, NT>;
    const size_t smem = RowTmaSmem<CV, NS, NT>::bytes(cfg.zseg);
    if (smem > 227 * 1024) return cudaSuccess;
    CUtensorMap tm_mid, tm_halo;
    if (!encode_row_box<R>(&tm_mid, a.in, a.P, a.SV, CV, G::WX)) return cudaSuccess;
    if (!encode_row_box<R>(&tm_halo, a.in, a.P, a.SV, CV, G::TX)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_apply_rowtma<R, CV, NS, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nchunks = (a.SV + CV - 1) / CV;
    const long long nblk = (long long)ntiles * nchunks;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_apply_rowtma<R, CV, NS, NT, MINB><<<(unsigned)nblk, dim3(CV, G::TX, G::TY), smem, st>>>(a, tm_mid, tm_halo,
                                                                                          nchunks);
    *launched = true;
    return cudaGetLastError();
}

// Row-TMA staged stencil (kernel 4) in the staged kernel's block shape with
// two vectors per point (cv = 2); *launched = false when it does not apply
// (no tensor-map encoder, another cv, too much shared memory).
template <typename R>
cudaError_t launch_apply_rowtma(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                                bool *launched) {
    *launched = false;
    if (ntiles == 0 || a.err == nullptr || (long long)a.P * a.SV >= 0x7fffffffLL) return cudaSuccess;
    int cv, nxr, ty;
    stage_shape(cfg, a.SV, &cv, &nxr, &ty);
    if (cv != 2) return cudaSuccess;
    if constexpr (sizeof(R) == 8) {
        // complex128 is bound by FP64 arithmetic: one shape (the tiles were
        // built for cfg.threads, so other shapes fall back to kernel 0)
        if (cfg.threads == 512) return cudaSuccess;
        return launch_rowtma_t<R, 2, 4, 256, 2>(a, cfg, ntiles, st, launched);
    } else {
        if (cfg.threads == 512) return launch_rowtma_t<R, 2, 6, 512, 1>(a, cfg, ntiles, st, launched);
        if (cfg.stages >= 5) return launch_rowtma_t<R, 2, 5, 256, 2>(a, cfg, ntiles, st, launched);
        return launch_rowtma_t<R, 2, 4, 256, 2>(a, cfg, ntiles, st, launched);
    }
}

// ------------------------------------------------------------- batches ---
// One launch per Horner stage for many independent complex64 systems: the
// stencil takes (system, tile, chunk) work items (k_batch_quad, rsg_quad.cu);
// projector coefficients, their reduction and the projector scatter are
// batched the same way here.
#if !defined(RSG_ONLY_DOUBLE) && !defined(RSG_ROWTMA_TU)

// <p_ai|u> partial sums over one sphere chunk of one system (block 8 x 32).
template <int NP>
__global__ void __launch_bounds__(256) k_batch_proj_dot(const SysArgs *__restrict__ sys,
                                                        const BWork *__restrict__ work, int in_c) {
    using V = VT<float>;
    using T = float4;
    __shared__ double red[256 * 4];
    const BWork w = work[blockIdx.x];
    const SysArgs &S = sys[w.sys];
    const int c = w.a, v = threadIdx.x, SV = S.SV;
    const T *u = (const T *)S.vec[in_c];
    const int q0 = S.chunk_q0[c], q1 = S.chunk_q1[c];
    T acc[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) acc[i] = V::zero();
    if (v < SV) {
        // four entries per iteration (independent loads in flight together)
        const int by = blockDim.y;
        int q = q0 + threadIdx.y;
        for (; q + 3 * by < q1; q += 4 * by) {
            int pt[4];
#pragma unroll
            for (int k = 0; k < 4; k++) pt[k] = S.q_pt[q + k * by];
            T val[4];
#pragma unroll
            for (int k = 0; k < 4; k++) val[k] = V::ldg(u + pt[k] * SV + v);
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int i = 0; i < NP; i++) V::fma(acc[i], S.q_p[(q + k * by) * NP + i], val[k]);
        }
        for (; q < q1; q += by) {
            const T val = V::ldg(u + S.q_pt[q] * SV + v);
#pragma unroll
            for (int i = 0; i < NP; i++) V::fma(acc[i], S.q_p[q * NP + i], val);
        }
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i = 0; i < NP; i++) {
        red[tid * 4 + 0] = acc[i].x;
        red[tid * 4 + 1] = acc[i].y;
        red[tid * 4 + 2] = acc[i].z;
        red[tid * 4 + 3] = acc[i].w;
        __syncthreads();
        if (threadIdx.y == 0 && v < SV) {
            double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            for (int l = 0; l < (int)blockDim.y; l++) {
                const double *r = red + (l * blockDim.x + threadIdx.x) * 4;
                s0 += r[0];
                s1 += r[1];
                s2 += r[2];
                s3 += r[3];
            }
            double *dst = S.partial + (((int64_t)c * NP + i) * SV + v) * 4;
            dst[0] = s0;
            dst[1] = s1;
            dst[2] = s2;
            dst[3] = s3;
        }
        __syncthreads();
    }
}

// D[a, i, s] = sum_j h_a[i][j] h^3 sum_chunks partial  (one block per (sys, atom))
__global__ void k_batch_proj_reduce(const SysArgs *__restrict__ sys, const BWork *__restrict__ work) {
    const BWork w = work[blockIdx.x];
    const SysArgs &S = sys[w.sys];
    const int a = w.a, s = threadIdx.x, ldc = 2 * S.SV, npmax = S.npmax;
    if (s >= ldc) return;
    double cr[9], ci[9];
    for (int i = 0; i < npmax; i++) {
        double sr = 0.0, si = 0.0;
        for (int c = S.atom_chunk0[a]; c < S.atom_chunk0[a + 1]; c++) {
            const double *p = S.partial + (((int64_t)c * npmax + i) * ldc + s) * 2;
            sr += p[0];
            si += p[1];
        }
        cr[i] = S.h3 * sr;
        ci[i] = S.h3 * si;
    }
    for (int i = 0; i < npmax; i++) {
        double dr = 0.0, di = 0.0;
        for (int j = 0; j < npmax; j++) {
            const double hij = S.hm[((int64_t)a * npmax + i) * npmax + j];
            dr += hij * cr[j];
            di += hij * ci[j];
        }
        float *dst = S.D + (((int64_t)a * npmax + i) * ldc + s) * 2;
        dst[0] = (float)dr;
        dst[1] = (float)di;
    }
}

cudaError_t launch_batch_proj(const SysArgs *sys, const BWork *dot_work, int ndot, const BWork *red_work,
                              int nred, int in_c, int npmax, cudaStream_t st) {
    if (ndot == 0) return cudaSuccess;
    switch (npmax) {
    case 1: k_batch_proj_dot<1><<<ndot, dim3(8, 32), 0, st>>>(sys, dot_work, in_c); break;
    case 4: k_batch_proj_dot<4><<<ndot, dim3(8, 32), 0, st>>>(sys, dot_work, in_c); break;
    case 9: k_batch_proj_dot<9><<<ndot, dim3(8, 32), 0, st>>>(sys, dot_work, in_c); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_batch_proj_reduce<<<nred, 32, 0, st>>>(sys, red_work);
    return cudaGetLastError();
}

// out += alpha * projector terms at up to 32 union points of one system.
__global__ void __launch_bounds__(256) k_batch_scatter(const SysArgs *__restrict__ sys,
                                                       const BWork *__restrict__ work, int out_c, float ar,
                                                       float ai) {
    using V = VT<float>;
    using T = float4;
    const BWork w = work[blockIdx.x];
    const SysArgs &S = sys[w.sys];
    const int u = w.a + threadIdx.y, v = threadIdx.x, SV = S.SV;
    if (u >= S.nu || u >= w.a + w.b || v >= SV) return;
    const int p = S.u_pts[u];
    const T *D = (const T *)S.D;
    T sum = V::zero();
    for (int e = S.u_ptr[u]; e < S.u_ptr[u + 1]; e++) {
        const int at = S.e_atom[e];
        const float *pv = S.e_p + e * S.npmax;
        const T *Da = D + at * S.npmax * SV + v;
        for (int i = 0; i < S.npmax; i++) V::fma(sum, pv[i], Da[i * SV]);
    }
    T *out = (T *)S.vec[out_c];
    const int o = p * SV + v;
    out[o] = V::add(out[o], V::cmul(ar, ai, sum));
}

cudaError_t launch_batch_scatter(const SysArgs *sys, const BWork *work, int nwork, int out_c, float ar,
                                 float ai, cudaStream_t st) {
    if (nwork == 0) return cudaSuccess;
    k_batch_scatter<<<nwork, dim3(8, 32), 0, st>>>(sys, work, out_c, ar, ai);
    return cudaGetLastError();
}
#endif

#if defined(RSG_ROWTMA_TU)
// the complex64 row-TMA kernels compile in a translation unit of their own
template cudaError_t launch_apply_rowtma<float>(const ApplyArgs<float> &, const TileCfg &, int, cudaStream_t, bool *);
#elif !defined(RSG_ONLY_DOUBLE)
template cudaError_t launch_apply_tma<float>(const ApplyArgs<float> &, const TileCfg &, int, cudaStream_t, bool *);
template cudaError_t launch_apply<float>(const ApplyArgs<float> &, const TileCfg &, int, cudaStream_t);
template cudaError_t launch_apply_naive_odd<float>(const ApplyArgs<float> &, cudaStream_t);
template cudaError_t launch_proj_dot<float>(const void *, int, const ProjDev &, double *, cudaStream_t);
template cudaError_t launch_proj_coeffs<float>(const void *, int, const ProjDev &, double *, unsigned *, double,
                                               void *, cudaStream_t);
template cudaError_t launch_proj_reduce<float>(const double *, int, const ProjDev &, double, void *, cudaStream_t);
template cudaError_t launch_proj_scatter<float>(const ApplyArgs<float> &, const ProjDev &, cudaStream_t);
#endif
#ifndef RSG_ONLY_FLOAT
template cudaError_t launch_apply_tma<double>(const ApplyArgs<double> &, const TileCfg &, int, cudaStream_t, bool *);
template cudaError_t launch_apply_rowtma<double>(const ApplyArgs<double> &, const TileCfg &, int, cudaStream_t, bool *);
template cudaError_t launch_apply<double>(const ApplyArgs<double> &, const TileCfg &, int, cudaStream_t);
template cudaError_t launch_apply_naive_odd<double>(const ApplyArgs<double> &, cudaStream_t);
template cudaError_t launch_proj_dot<double>(const void *, int, const ProjDev &, double *, cudaStream_t);
template cudaError_t launch_proj_coeffs<double>(const void *, int, const ProjDev &, double *, unsigned *, double,
                                                void *, cudaStream_t);
template cudaError_t launch_proj_reduce<double>(const double *, int, const ProjDev &, double, void *, cudaStream_t);
template cudaError_t launch_proj_scatter<double>(const ApplyArgs<double> &, const ProjDev &, cudaStream_t);
#endif

}  // namespace rsg
