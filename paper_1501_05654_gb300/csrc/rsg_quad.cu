// Register-blocked staged stencil for complex64 blocks (kernel 5).
//
// The operator and epilogue are those of rsg_kernels.cu (8th-order 25-point
// star Laplacian with zero values outside the mesh, local potential and
// dipole field on the diagonal, arXiv:1501.05654 Sec. 1 and Sec.
// "Parallelization, optimizations and graphics processing units"); projector terms are added afterwards by k_proj_scatter.
//
// k_apply_quad: the z-march of k_apply_staged with register blocking.  A
// block owns a 16 x TY tile of points and one 32-byte chunk of each point's
// states (four complex64 values).  A thread owns one of those four values at
// a 2 x 2 group of points (x0, x0 + 1) x (y0, y0 + 1) and keeps four
// nine-deep z queues.  Per plane it reads two x windows of ten points and two
// y columns of eight more: 36 eight-byte shared-memory loads for four
// outputs (9 per output, 72 bytes), against 17 sixteen-byte loads per two
// outputs in k_apply_staged (136 bytes per output); the wider tile also cuts
// the halo fill from 2.5x to 2.0x (TY = 16) or 2.17x (TY = 12).
//
// Shared-memory slot of one plane: (TY + 8) rows x 24 columns of 32-byte
// point records; within a row the even x columns come first and the odd ones
// second, so that for a fixed offset the x-adjacent threads of a warp read
// consecutive records (no bank conflicts).  Planes stream through NS slots
// filled with cp.async (ghost points zero-filled), one block barrier per
// plane, as in k_apply_staged; the potential of each interior point and the
// base value of each output travel with the plane that uses them.
//
// Complex scaling (CS = true): the diagonal is the complex v_theta e^{2i theta}
// of each point (staged like V, 8 bytes per point) and the caller folds the
// kinetic rotation e^{-2i theta} into alpha, so the rest of the kernel is the
// same.
#include <cuda.h>

#include "rsg_async.cuh"
#include "rsg_batch.cuh"
#include "rsg_internal.h"
#include "rsg_vec.cuh"

namespace rsg {

template <int NYT>
struct QuadGeom {
    static constexpr int NXT = 8, NC = 4;                  // x threads, complex values per record
    static constexpr int NT = NC * NXT * NYT;              // threads
    static constexpr int TX = 2 * NXT, TY = 2 * NYT;       // tile
    static constexpr int WX = TX + 8, WY = TY + 8, HW = WX / 2;
    // the star stencil reads a cross: the TY middle rows at full width and
    // four rows above and below at the interior width
    static constexpr int NMID = TY * WX, NCROSS = NMID + 8 * TX;
    static constexpr int SLOT = WY * WX * NC;              // float2 entries per plane
    static constexpr int NPTS = TX * TY;                   // interior points
    static_assert(NPTS == NT, "one interior point per thread for the potential");
};

// slot column of window column xx (even columns first, then odd)
__host__ __device__ constexpr int qcol(int xx, int hw) { return (xx >> 1) + (xx & 1) * hw; }

template <int NYT>
struct QCtx {
    const float2 *slots;
    const float2 *bslots;
    const float *vslots;
    const SRow *srows;
    int woff;          // float2 offset of window column 0 of row y0 in a slot
    int boff, voff;    // this thread's first base / potential entry in a slot
    int yrow;          // row-table row of y0 (4 + 2 yt)
    int x0, k, zbase, zlo, zhi, zc0, zc1, ld;
    bool vok;
    float fxy[4];      // f0 + fx x + fy y of the four points
};

// Bounded mbarrier wait (the pipelined variants): false after 2^22 polls.
constexpr long kQuadWaitLimit = 1L << 22;
__device__ __forceinline__ bool qbar_wait(unsigned bar, unsigned parity) {
    for (long it = 0; it < kQuadWaitLimit; ++it) {
        unsigned ok;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// y = alpha * acc + beta * base; out = y; optional acc += gamma * y
__device__ __forceinline__ void finish_quad(const ApplyArgs<float> &a, int o, float2 acc, float2 bv) {
    float2 y = f2_fma(make_float2(-a.ai, a.ai), make_float2(acc.y, acc.x), f2_mul(make_float2(a.ar, a.ar), acc));
    if (a.base != nullptr) {
        y = f2_fma(make_float2(a.br, a.br), bv, y);
        y = f2_fma(make_float2(-a.bi, a.bi), make_float2(bv.y, bv.x), y);
    }
    ((float2 *)a.out)[o] = y;
    if (a.acc != nullptr) {
        float2 s = a.acc_base != nullptr ? ((const float2 *)a.acc_base)[o] : ((float2 *)a.acc)[o];
        s = f2_fma(make_float2(a.gr, a.gr), y, s);
        s = f2_fma(make_float2(-a.gi, a.gi), make_float2(y.y, y.x), s);
        ((float2 *)a.acc)[o] = s;
    }
}

// Plane j has landed: add its contributions to the four queues and retire
// the outputs of plane j - 4.  Entry k of a queue holds output plane
// j - 4 + k; every entry takes exactly one update per plane, and each update
// is written one entry down, so the queue shifts without extra moves and the
// loop body exists once (no unrolling for register renaming, which kept the
// code out of the instruction cache).
template <int NYT, int NS, bool CS>
__device__ __forceinline__ void quad_plane(const ApplyArgs<float> &a, const QCtx<NYT> &c, int j,
                                           float2 (&q)[4][9]) {
    using G = QuadGeom<NYT>;
    constexpr int RW = G::WX * G::NC;     // one slot row, float2 entries
    const int sl = j % NS;
    const float2 *pw = c.slots + sl * G::SLOT + c.woff;
    // window column k (x = x0 - 4 + k) of row r (y = y0 + r)
#define QW(r, k) pw[(r) * RW + (((k) >> 1) + ((k) & 1) * G::HW) * G::NC]
    const int p = c.zbase + j;
    const float2 w1 = make_float2(a.w[1], a.w[1]), w2 = make_float2(a.w[2], a.w[2]);
    const float2 w3 = make_float2(a.w[3], a.w[3]), w4 = make_float2(a.w[4], a.w[4]);
    // points 0 = (x0, y0), 1 = (x0+1, y0), 2 = (x0, y0+1), 3 = (x0+1, y0+1)
    float2 s[4], cen[4];
    if (p >= c.zc0 && p <= c.zc1) {
#pragma unroll
        for (int r = 0; r < 2; r++) {
            float2 W[10];
#pragma unroll
            for (int k = 0; k < 10; k++) W[k] = QW(r, k);
            cen[2 * r] = W[4];
            cen[2 * r + 1] = W[5];
            float2 t = f2_mul(w1, f2_add(W[3], W[5]));
            t = f2_fma(w2, f2_add(W[2], W[6]), t);
            t = f2_fma(w3, f2_add(W[1], W[7]), t);
            s[2 * r] = f2_fma(w4, f2_add(W[0], W[8]), t);
            t = f2_mul(w1, f2_add(W[4], W[6]));
            t = f2_fma(w2, f2_add(W[3], W[7]), t);
            t = f2_fma(w3, f2_add(W[2], W[8]), t);
            s[2 * r + 1] = f2_fma(w4, f2_add(W[1], W[9]), t);
        }
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
            // rows y0 - 4 .. y0 - 1 and y0 + 2 .. y0 + 5 of column x0 + dx
            const float2 m4 = QW(-4, 4 + dx), m3 = QW(-3, 4 + dx), m2 = QW(-2, 4 + dx), m1 = QW(-1, 4 + dx);
            const float2 p2 = QW(2, 4 + dx), p3 = QW(3, 4 + dx), p4 = QW(4, 4 + dx), p5 = QW(5, 4 + dx);
            float2 t = f2_fma(w1, f2_add(m1, cen[2 + dx]), s[dx]);
            t = f2_fma(w2, f2_add(m2, p2), t);
            t = f2_fma(w3, f2_add(m3, p3), t);
            s[dx] = f2_fma(w4, f2_add(m4, p4), t);
            t = f2_fma(w1, f2_add(cen[dx], p2), s[2 + dx]);
            t = f2_fma(w2, f2_add(m1, p3), t);
            t = f2_fma(w3, f2_add(m2, p4), t);
            s[2 + dx] = f2_fma(w4, f2_add(m3, p5), t);
        }
        if constexpr (CS) {
            // complex diagonal v_theta e^{2i theta} plus the stencil's real
            // centre weight (no field terms under complex scaling)
            const float2 *vv = (const float2 *)c.vslots + sl * G::NPTS + c.voff;
            const float w0 = 3.0f * a.w[0];
#pragma unroll
            for (int pt = 0; pt < 4; pt++) {
                const float2 d = vv[(pt >> 1) * G::TX + (pt & 1)];
                const float dr = d.x + w0;
                s[pt] = f2_fma(make_float2(dr, dr), cen[pt], s[pt]);
                s[pt] = f2_fma(make_float2(-d.y, d.y), make_float2(cen[pt].y, cen[pt].x), s[pt]);
            }
        } else {
            const float fz = a.fz * (float)p + 3.0f * a.w[0];
            const float *vv = c.vslots + sl * G::NPTS + c.voff;
#pragma unroll
            for (int pt = 0; pt < 4; pt++) {
                // diagonal: staged V (zero outside the mesh, where the value is zero too)
                const float d = vv[(pt >> 1) * G::TX + (pt & 1)] + c.fxy[pt] + fz;
                s[pt] = f2_fma(make_float2(d, d), cen[pt], s[pt]);
            }
        }
    } else {
        // no mesh point in the thread's columns at this plane: nothing to add
#pragma unroll
        for (int pt = 0; pt < 4; pt++) s[pt] = cen[pt] = make_float2(0.f, 0.f);
    }
#undef QW
    float2 done[4];
#pragma unroll
    for (int pt = 0; pt < 4; pt++) {
        float2 *qq = q[pt];
        const float2 cv = cen[pt];
        done[pt] = f2_fma(w4, cv, qq[0]);     // output j - 4 is complete
        qq[0] = f2_fma(w3, cv, qq[1]);
        qq[1] = f2_fma(w2, cv, qq[2]);
        qq[2] = f2_fma(w1, cv, qq[3]);
        qq[3] = f2_add(qq[4], s[pt]);
        qq[4] = f2_fma(w1, cv, qq[5]);
        qq[5] = f2_fma(w2, cv, qq[6]);
        qq[6] = f2_fma(w3, cv, qq[7]);
        qq[7] = f2_fma(w4, cv, qq[8]);
        qq[8] = make_float2(0.f, 0.f);
    }
    const int zo = p - 4;
    if (zo >= c.zlo && zo < c.zhi && c.vok) {
        const SRow *ro = c.srows + (j - 4) * G::WY + c.yrow;
        const float2 *bb = c.bslots + sl * G::NPTS * G::NC + c.boff;
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const SRow rw = ro[dy];
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const int x = c.x0 + dx;
                if (x >= rw.xmin && x <= rw.xmax)
                    finish_quad(a, (rw.start + (x - rw.xmin)) * c.ld + c.k, done[2 * dy + dx],
                                bb[(dy * G::TX + dx) * G::NC]);
            }
        }
    }
}

// SYNC selects how a plane's slot is handed between its copies and its
// readers: 0 = one block barrier per plane; 1 and 2 = per-slot mbarriers, a
// "full" barrier that every thread's copies arrive on
// (cp.async.mbarrier.arrive.noinc) and an "empty" barrier that every warp
// arrives on after its last read of the plane.  With 1 the copies run NS - 1
// planes ahead (warps stay in step, like the barrier); with 2 they run NS - 2
// planes ahead and a warp may run one plane ahead of the slowest.
// One block of the register-blocked stencil: tile tl, four-value chunk
// `chunk` of the system described by a.  Shared by the single-system and
// batched kernels.
template <int NYT, int NS, int SYNC, bool CS = false>
__device__ __forceinline__ void quad_block(const ApplyArgs<float> &a, const Tile tl, const int chunk,
                                           unsigned char *smraw) {
    using G = QuadGeom<NYT>;
    constexpr int NT = G::NT, TX = G::TX, TY = G::TY, WX = G::WX, WY = G::WY, NC = G::NC;
    float2 *slots = (float2 *)smraw;                           // NS x SLOT
    float2 *bslots = slots + NS * G::SLOT;                     // NS x NPTS x NC
    float *vslots = (float *)(bslots + NS * G::NPTS * NC);     // NS x NPTS (x 2 with CS: complex)
    SRow *srows = (SRow *)(vslots + NS * G::NPTS * (CS ? 2 : 1));   // WY x np

    const int ny = a.ny, nz = a.nz, ld = 2 * a.SV;
    const int xbase = tl.tx * TX - 4, ybase = tl.ty * TY - 4, zbase = tl.zlo - 4;
    const int np = tl.zhi - tl.zlo + 8;
    const int cc = threadIdx.x, xt = threadIdx.y, yt = threadIdx.z;
    const int tid = (yt * G::NXT + xt) * NC + cc;
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
    // full / empty mbarriers of the NS slots, after the row table
    const unsigned bar0 =
        ((unsigned)__cvta_generic_to_shared(srows) + (unsigned)(WY * (tl.zhi - tl.zlo + 8) * sizeof(SRow)) + 7u) & ~7u;
    if constexpr (SYNC > 0) {
        if (tid == 0) {
            for (int k = 0; k < NS; k++) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * k), "r"(NT) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * (NS + k)), "r"(NYT)
                             : "memory");
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();

    const float2 *__restrict__ in2 = (const float2 *)a.in;
    const float2 *__restrict__ base2 = (const float2 *)a.base;
    const int k0 = NC * chunk;                                  // first complex value of the chunk
    const unsigned s_slots = (unsigned)__cvta_generic_to_shared(slots);
    const unsigned s_b = (unsigned)__cvta_generic_to_shared(bslots);
    const unsigned s_v = (unsigned)__cvta_generic_to_shared(vslots);
    const int pyy = tid / TX, pxx = tid - pyy * TX;              // this thread's potential point
    // plane j into slot j % NS: the cross of state records, the potential of
    // the interior points, and the base values of the outputs of plane j - 4.
    // A staging task is four x-adjacent points of one cross row, taken by two
    // adjacent threads, one 16-byte half of each record apiece (one row
    // lookup, four copies; the lanes of a warp still read whole 32-byte
    // sectors): TY x 6 tasks in the middle rows, 8 x 4 in the halo rows.
    constexpr int NTASK = TY * (WX / 4) + 8 * (TX / 4);
    const int hh = tid & 1;
    auto stage = [&](int j) {
        const int sl = j % NS;
        const SRow *rr = srows + j * WY;
        const unsigned dslot = s_slots + (unsigned)(sl * G::SLOT * 8 + hh * 16);
        const bool hok = k0 + 2 * hh < ld;
#pragma unroll
        for (int t0 = 0; t0 < 2 * NTASK; t0 += NT) {
            const int t = (t0 + tid) >> 1;
            if (t0 + NT <= 2 * NTASK || t < NTASK) {
                int yy, xx0;
                if (t < TY * (WX / 4)) {
                    yy = 4 + t / (WX / 4);
                    xx0 = 4 * (t - (yy - 4) * (WX / 4));
                } else {
                    const int t2 = t - TY * (WX / 4), r = t2 / (TX / 4);
                    yy = r < 4 ? r : TY + r;
                    xx0 = 4 + 4 * (t2 - r * (TX / 4));
                }
                const SRow rw = rr[yy];
                const unsigned drow = dslot + (unsigned)(yy * WX * NC * 8);
#pragma unroll
                for (int d = 0; d < 4; d++) {
                    const int x = xbase + xx0 + d;
                    const bool ok = (x >= rw.xmin) & (x <= rw.xmax) & hok;
                    const float2 *src = in2 + (ok ? (rw.start + (x - rw.xmin)) * ld + k0 + 2 * hh : 0);
                    cp_async16(drow + (unsigned)(qcol(xx0 + d, G::HW) * NC * 8), src, ok ? 16 : 0);
                }
            }
        }
        {
            const SRow rw = rr[4 + pyy];
            const int x = tl.tx * TX + pxx;
            const bool ok = (x >= rw.xmin) & (x <= rw.xmax);
            if constexpr (CS)
                cp_async_small<8>(s_v + (unsigned)((sl * G::NPTS + tid) * 8),
                                  (const float2 *)a.Vc + (ok ? rw.start + (x - rw.xmin) : 0), ok ? 8 : 0);
            else
                cp_async_small<4>(s_v + (unsigned)((sl * G::NPTS + tid) * 4),
                                  a.V + (ok ? rw.start + (x - rw.xmin) : 0), ok ? 4 : 0);
        }
        if (base2 != nullptr && j >= 4) {
            // base records of interior points 2 (tid / 2) and 2 (tid / 2) + 1
            // (same row), half hh of each
            const int pi0 = 2 * (tid >> 1), by = pi0 / TX, bx = pi0 - by * TX;
            const SRow rw = srows[(j - 4) * WY + 4 + by];
#pragma unroll
            for (int d = 0; d < 2; d++) {
                const int x = tl.tx * TX + bx + d;
                const bool ok = (x >= rw.xmin) & (x <= rw.xmax) & hok;
                const float2 *src = base2 + (ok ? (rw.start + (x - rw.xmin)) * ld + k0 + 2 * hh : 0);
                cp_async16(s_b + (unsigned)(((sl * G::NPTS + pi0 + d) * NC + 2 * hh) * 8), src, ok ? 16 : 0);
            }
        }
    };

    QCtx<NYT> c;
    c.slots = slots;
    c.bslots = bslots;
    c.vslots = vslots;
    c.srows = srows;
    c.woff = ((4 + 2 * yt) * WX + xt) * NC + cc;
    c.boff = ((2 * yt) * TX + 2 * xt) * NC + cc;
    c.voff = (2 * yt) * TX + 2 * xt;
    c.yrow = 4 + 2 * yt;
    c.x0 = tl.tx * TX + 2 * xt;
    c.k = k0 + cc;
    c.vok = c.k < ld;
    c.ld = ld;
    c.zbase = zbase;
    c.zlo = tl.zlo;
    c.zhi = tl.zhi;
    const int y0 = tl.ty * TY + 2 * yt;
#pragma unroll
    for (int pt = 0; pt < 4; pt++)
        c.fxy[pt] = a.f0 + a.fx * (float)(c.x0 + (pt & 1)) + a.fy * (float)(y0 + (pt >> 1));
    // planes where any of the thread's four columns has points
    c.zc0 = 1 << 30;
    c.zc1 = -(1 << 30);
    for (int jj = 0; jj < np; jj++) {
        const SRow r0 = srows[jj * WY + 4 + 2 * yt], r1 = srows[jj * WY + 5 + 2 * yt];
        const bool on = (c.x0 + 1 >= r0.xmin && c.x0 <= r0.xmax) || (c.x0 + 1 >= r1.xmin && c.x0 <= r1.xmax);
        if (on) {
            c.zc0 = min(c.zc0, zbase + jj);
            c.zc1 = max(c.zc1, zbase + jj);
        }
    }
    float2 q[4][9];
#pragma unroll
    for (int pt = 0; pt < 4; pt++)
#pragma unroll
        for (int k = 0; k < 9; k++) q[pt][k] = make_float2(0.f, 0.f);

    if constexpr (SYNC == 0) {
#pragma unroll 1
        for (int j = 0; j < NS - 1; j++) {
            if (j < np) stage(j);
            cp_async_commit();
        }
        // plane j has landed for every thread after the barrier; the slot then
        // refilled (plane j + NS - 1) was last read at plane j - 1
#pragma unroll 1
        for (int j = 0; j < np; j++) {
            cp_async_wait<NS - 2>();
            __syncthreads();
            if (j + NS - 1 < np) stage(j + NS - 1);
            cp_async_commit();
            quad_plane<NYT, NS, CS>(a, c, j, q);
        }
        cp_async_wait<0>();
    } else {
        constexpr int D = SYNC == 1 ? NS - 1 : NS - 2;     // planes the copies run ahead
        const unsigned full0 = bar0, empty0 = bar0 + 8 * NS;
        const int lane = tid & 31;
        int bad = 0;
        auto arrive_full = [&](int p) {
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full0 + 8 * (p % NS))
                         : "memory");
        };
#pragma unroll 1
        for (int j = 0; j < D && j < np; j++) {
            stage(j);
            arrive_full(j);
        }
#pragma unroll 1
        for (int j = 0; j < np; j++) {
            const int pn = j + D;
            if (pn < np) {
                // slot of plane pn last held plane pn - NS: every warp has read it
                if (pn >= NS && !qbar_wait(empty0 + 8 * (pn % NS), (unsigned)((pn / NS - 1) & 1))) bad = 1;
                stage(pn);
                arrive_full(pn);
            }
            if (!qbar_wait(full0 + 8 * (j % NS), (unsigned)((j / NS) & 1))) bad = 1;
            quad_plane<NYT, NS, CS>(a, c, j, q);
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty0 + 8 * (j % NS)) : "memory");
        }
        cp_async_wait<0>();
        // every copy has landed and every full phase up to plane np - 1 was
        // waited on, so no arrival is left in flight when the block leaves
        if (bad) atomicExch(a.err, 2);
    }
}

template <int NYT, int NS, int MINB, int SYNC, bool CS = false>
__global__ void __launch_bounds__(QuadGeom<NYT>::NT, MINB) k_apply_quad(const ApplyArgs<float> a, int nchunks) {
    extern __shared__ __align__(128) unsigned char smraw[];
    quad_block<NYT, NS, SYNC, CS>(a, a.tiles[blockIdx.x / nchunks], blockIdx.x % nchunks, smraw);
}

// Batches: every block takes a (system, tile, chunk) work item and runs the
// register-blocked block for that system (16 x 12 tiles, 192 threads).
__global__ void __launch_bounds__(QuadGeom<kBatchTY / 2>::NT, 2)
    k_batch_quad(const SysArgs *__restrict__ sys, const BWork *__restrict__ work, int in_c, int out_c, float ar,
                 float ai) {
    extern __shared__ __align__(128) unsigned char smraw[];
    const BWork w = work[blockIdx.x];
    const SysArgs &S = sys[w.sys];
    const ApplyArgs<float> a = batch_args(S, in_c, out_c, ar, ai);
    quad_block<kBatchTY / 2, 4, 0>(a, S.tiles[w.a], w.b, smraw);
}

// Tile of kernel 5: 16 x 16 points with 256 threads, 16 x 10 with 160
// (three blocks per SM at up to 136 registers), 16 x 12 otherwise (192
// threads, two blocks per SM at up to 170 registers).
void quad_shape(const TileCfg &cfg, int *TX, int *TY) {
    *TX = 16;
    *TY = cfg.threads == 256 ? 16 : cfg.threads == 160 ? 10 : 12;
}

size_t quad_smem_bytes(int nyt, int ns, int zseg, bool cs = false) {
    const size_t nt = 32 * (size_t)nyt, wy = 2 * (size_t)nyt + 8;
    // slots, base and potential rings (complex potential with cs), row
    // table, then 2 NS mbarriers
    return (size_t)ns * (wy * 24 * 4 * 8 + nt * 4 * 8 + nt * 4 * (cs ? 2 : 1)) + wy * (zseg + 8) * sizeof(SRow) + 8 +
           16 * (size_t)ns;
}

template <int NYT, int NS, int MINB, int SYNC, bool CS = false>
static cudaError_t launch_quad_t(const ApplyArgs<float> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                                 bool *launched) {
    using G = QuadGeom<NYT>;
    const size_t smem = quad_smem_bytes(NYT, NS, cfg.zseg, CS);
    if (smem > 227 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_apply_quad<NYT, NS, MINB, SYNC, CS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nchunks = (2 * a.SV + G::NC - 1) / G::NC;
    const long long nblk = (long long)ntiles * nchunks;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_apply_quad<NYT, NS, MINB, SYNC, CS><<<(unsigned)nblk, dim3(G::NC, G::NXT, NYT), smem, st>>>(a, nchunks);
    *launched = true;
    return cudaGetLastError();
}

cudaError_t launch_batch_stencil(const SysArgs *sys, const BWork *work, int nwork, int in_c, int out_c,
                                 float ar, float ai, cudaStream_t st) {
    if (nwork == 0) return cudaSuccess;
    using G = QuadGeom<kBatchTY / 2>;
    static_assert(G::TX == kBatchNXR && G::TY == kBatchTY && G::NC == 2 * kBatchCV,
                  "batch tiles and chunks must match the block geometry");
    const size_t smem = quad_smem_bytes(kBatchTY / 2, 4, kBatchZseg);
    cudaError_t e = cudaFuncSetAttribute(k_batch_quad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_quad<<<nwork, dim3(G::NC, G::NXT, kBatchTY / 2), smem, st>>>(sys, work, in_c, out_c, ar, ai);
    return cudaGetLastError();
}

cudaError_t launch_apply_quad(const ApplyArgs<float> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                              bool *launched) {
    *launched = false;
    // complex offsets are 32-bit: P * ld < 2^31
    if (ntiles == 0 || (long long)a.P * 2 * a.SV >= 0x7fffffffLL) return cudaSuccess;
    if (a.err == nullptr && cfg.sync != 0) return cudaSuccess;
    if (a.Vc != nullptr) {
        // complex scaling: the default block shape (16 x 12 tiles, 3 slots) only
        if (cfg.threads == 256 || cfg.threads == 160 || cfg.sync != 0 || cfg.stages != 3) return cudaSuccess;
        return launch_quad_t<6, 3, 2, 0, true>(a, cfg, ntiles, st, launched);
    }
    if (cfg.threads == 256) return launch_quad_t<8, 3, 2, 0>(a, cfg, ntiles, st, launched);
    if (cfg.threads == 160) return launch_quad_t<5, 3, 3, 0>(a, cfg, ntiles, st, launched);
    switch (cfg.sync) {
    case 1: return launch_quad_t<6, 4, 2, 1>(a, cfg, ntiles, st, launched);
    case 2: return launch_quad_t<6, 4, 2, 2>(a, cfg, ntiles, st, launched);
    default:
        if (cfg.stages == 3) return launch_quad_t<6, 3, 2, 0>(a, cfg, ntiles, st, launched);
        return launch_quad_t<6, 4, 2, 0>(a, cfg, ntiles, st, launched);
    }
}

}  // namespace rsg
