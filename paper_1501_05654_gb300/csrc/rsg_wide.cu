// Warp-specialised stencil for complex64 blocks (kernel 7).
//
// The operator and epilogue are those of the other stencil kernels: the
// 8th-order 25-point star Laplacian with zero values outside the mesh, and
// the local potential and dipole field on the diagonal (arXiv:1501.05654
// Sec. 1 and Sec. "Parallelization, optimizations and graphics processing
// units"); projector terms are added afterwards by k_proj_scatter.
//
// A block owns a 16 x TY tile of (x, y) columns, marched along z, and one
// 128-byte chunk of every point's state row (16 complex64 values, the
// "record" of the point).
//
// One producer warp moves each plane into shared memory with 2-D tensor
// copies.  The copies view the state block as (points, state floats), and a
// mesh row is a run of consecutive point indices.  So each row of the plane's
// cross-shaped window is one box of 24 (or 16) records, or a few boxes of 16,
// 8, 4, 2 and 1 records where the mesh row covers only part of the window.
// Window positions outside the mesh must read zero.  They are filled by
// boxes placed wholly before point 0, which the copy engine fills with zeros.
// A position is re-zeroed only if it held a mesh point the last time its slot
// was used.  The base values of the plane's outputs (16-record boxes) and the
// potential (4-byte cp.async) travel in the same slot.
//
// Synchronisation uses two mbarriers per slot. The "full" barrier completes
// on the expected byte count plus the potential's cp.async arrivals. The
// "empty" barrier takes one arrival from each compute warp after its last
// read of the slot. No block-wide barrier runs inside the march.
//
// Compute warps (4 NYP of them): a thread owns one complex value of the chunk
// at a 2 x 2 group of points and keeps four nine-deep z queues, as in the
// register-blocked kernel 5.  A warp covers 4 x 2 columns.  Planes before the
// first mesh point of its columns, and after its last output, are passed with
// a wait and a release only.
//
// Every mbarrier wait is bounded.  A wait that gives up sets a block-wide
// abort flag.  Later waits then return at once, the producer stops issuing,
// and the block records status 2 (RSG_ERR_TIMEOUT) before it leaves.  The
// producer first waits, again with a bound, for the copies it has issued.
#include <cuda.h>

#include <array>
#include <mutex>
#include <unordered_map>

#include "rsg_async.cuh"
#include "rsg_internal.h"
#include "rsg_vec.cuh"

namespace rsg {

template <int NYP, int NPW = 1>
struct WideGeom {
    static constexpr int TX = 16, TY = 2 * NYP;
    static constexpr int WX = TX + 8, WY = TY + 8;   // window (cross inside the rectangle)
    static constexpr int NC = 16;                    // complex values per record
    static constexpr int REC = NC * 8;               // bytes per record
    static constexpr int NCW = 4 * NYP;              // compute warps
    static constexpr int NT = 32 * (NCW + NPW);      // plus the producer warps
    static constexpr int SLOT = WY * WX;             // records per plane
    static constexpr int NPTS = TX * TY;             // interior points
    static_assert(WY + TY <= 32 * NPW, "one producer lane per window row and per base row");
    static_assert((TX * TY) % 32 == 0, "the potential's points in groups of 32");
};

// Tensor maps of one launch, one per box width: u[w - 1] copies w = 1 .. 24
// records of the input block, b[w - 1] w = 1 .. 16 records of the base block,
// so that every run of consecutive records is a single copy.
struct WideMaps {
    CUtensorMap u[24];
    CUtensorMap b[16];
};

// Each poll suspends the thread until the phase completes or about 2 us
// pass; 2^20 polls bound a wait at about 2 s.
constexpr long kWideWaitLimit = 1L << 20;
constexpr unsigned kWideSuspendNs = 2000;
constexpr int kWideZeroPoint = -64;   // first point of a zero-fill box (every row out of range)

__device__ __forceinline__ bool wide_wait(unsigned bar, unsigned parity, volatile int *abort_flag) {
    for (long it = 0; it < kWideWaitLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(kWideSuspendNs)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void wide_box(unsigned dst, const CUtensorMap *tm, int c0, int p0, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(tm), "r"(c0), "r"(p0), "r"(bar)
        : "memory");
}

// y = alpha * acc + beta * base; out = y; optional acc += gamma * y
__device__ __forceinline__ void wide_finish(const ApplyArgs<float> &a, int o, float2 acc, float2 bv) {
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

// EPI 1: Horner stage, out = (i ai) H u + base (ar = 0, beta = 1, no
// accumulator); EPI 2: the same with a complex alpha (complex scaling's
// rotated Horner stage); EPI 0: the general epilogue of wide_finish.  CS 1: complex
// scaling, the diagonal is the complex a.Vc per point (v_theta e^{2i theta},
// interleaved) plus the stencil's real centre weight; the caller folds the
// kinetic rotation e^{-2i theta} into alpha and sets no field.
template <int NYP, int NS, int NPW, int EPI, int CS = 0>
__global__ void __launch_bounds__(WideGeom<NYP, NPW>::NT, 1)
    k_apply_wide(const ApplyArgs<float> a, int nchunks, const __grid_constant__ WideMaps maps) {
    using G = WideGeom<NYP, NPW>;
    constexpr int TX = G::TX, TY = G::TY, WX = G::WX, WY = G::WY, NC = G::NC, NCW = G::NCW;
    extern __shared__ __align__(128) unsigned char smraw[];
    // 1024-byte aligned start: u ring, base ring, potential ring, row table,
    // barriers, abort flag
    const unsigned sraw = (unsigned)__cvta_generic_to_shared(smraw);
    const unsigned s_u = (sraw + 1023u) & ~1023u;
    unsigned char *gbase = smraw + (s_u - sraw);
    const unsigned s_b = s_u + NS * G::SLOT * G::REC;
    const unsigned s_v = s_b + NS * G::NPTS * G::REC;
    constexpr int VBY = CS ? 8 : 4;   // bytes of the staged diagonal per point
    const Tile tl = a.tiles[blockIdx.x / nchunks];
    const int chunk = blockIdx.x % nchunks;
    const int np = tl.zhi - tl.zlo + 8;
    // window rows (producers) and tile rows (all warps) of every plane
    SRow *srows = (SRow *)(gbase + (s_v - s_u) + NS * G::NPTS * VBY);
    int2 *orows = (int2 *)(srows + WY * np);
    const unsigned s_rows = s_v + NS * G::NPTS * VBY;
    const unsigned bar0 = (s_rows + (unsigned)(WY * np * sizeof(SRow) + TY * np * sizeof(int2)) + 7u) & ~7u;
    volatile int *abort_flag = (volatile int *)(gbase + (bar0 - s_u) + 16 * NS);

    const int ny = a.ny, nz = a.nz, ld = 2 * a.SV;
    const int tx0 = tl.tx * TX, ty0 = tl.ty * TY;
    const int xb = tx0 - 4, ybase = ty0 - 4, zbase = tl.zlo - 4;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll 4
    for (int i = tid; i < WY * np; i += G::NT) {
        const int zz = i / WY;
        const int yy = ybase + (i - zz * WY);
        const int zg = zbase + zz;
        // start holds the point index of bbox column 0 of the row (start -
        // xmin), so that point (x, row) is start + x
        SRow r{0, 1, 0};
        if (yy >= 0 && yy < ny && zg >= 0 && zg < nz) {
            const Row g = a.rows[zg * ny + yy];
            r.start = g.start - g.xmin;
            r.xmin = (int16_t)g.xmin;
            r.xmax = (int16_t)g.xmax;
        }
        srows[i] = r;
    }
    // per plane and tile row: the point of bbox column 0 and a mask of the
    // tile columns that are mesh points
#pragma unroll 4
    for (int i = tid; i < TY * np; i += G::NT) {
        const int zz = i / TY;
        const int yy = ty0 + (i - zz * TY);
        const int zg = zbase + zz;
        int2 e = make_int2(0, 0);
        if (yy < ny && zg >= 0 && zg < nz) {
            const Row g = a.rows[zg * ny + yy];
            const int lo = max(g.xmin - tx0, 0), hi = min(g.xmax - tx0, TX - 1);
            e.x = g.start - g.xmin;
            e.y = lo <= hi ? (int)(((2u << hi) - 1u) & ~((1u << lo) - 1u)) : 0;
        }
        orows[i] = e;
    }
    __syncthreads();
    // Only planes [j0, j1] are staged: from the first plane with a point in
    // the tile's own columns to four planes past the last one (jl).  Planes
    // outside hold no value that reaches an output of the segment; the last
    // four carry only the base values of the outputs they complete.  Every
    // warp computes the same range.
    int jf = np, jl = -1;
    for (int jj = lane; jj < np; jj += 32) {
        int m = 0;
#pragma unroll
        for (int rr = 0; rr < TY; rr++) m |= orows[jj * TY + rr].y;
        if (m) {
            jf = min(jf, jj);
            jl = max(jl, jj);
        }
    }
    jf = __reduce_min_sync(0xffffffffu, jf);
    jl = __reduce_max_sync(0xffffffffu, jl);
    if (jl < 0) return;
    const int j0 = jf, j1 = min(np - 1, jl + 4);
    if (tid == 0) {
        for (int k = 0; k < NS; k++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * k), "r"(33 * NPW)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * (NS + k)), "r"(NCW)
                         : "memory");
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int k0 = NC * chunk;        // first complex value of the chunk
    const int c0 = 2 * k0;            // its float column in the tensor view

    if (warp >= NCW) {
        // ------------------------------------------------ producer warps
        // Row tasks of a plane: the WY window rows of the state block, then
        // the TY base rows of the outputs four planes back.  Lane l of
        // producer warp pw takes row task pw + NPW l.  The potential's points
        // are shared out in groups of 32.  Every lane first works out its
        // boxes; the boxes are then issued from one call site per pass, so
        // the issue loop runs once per box and not once per call site.
        const int pw = warp - NCW;
        const int r = pw + NPW * lane;
        const bool rowlane = r < WY;
        const bool baselane = a.base != nullptr && r >= WY && r < WY + TY;
        const int br = r - WY;
        const bool halo = r < 4 || r >= TY + 4;
        const int clo = halo ? 4 : 0, chi = halo ? 20 : 24;
        int pa[NS], pb[NS];   // window columns that held mesh points at the slot's last use
#pragma unroll
        for (int s = 0; s < NS; s++) {
            pa[s] = clo;
            pb[s] = chi;
        }
        int issued = 0;
        for (int q0 = 0; q0 <= j1 - j0; q0 += NS) {
#pragma unroll
            for (int s = 0; s < NS; s++) {
                const int q = q0 + s, j = j0 + q;   // q: staged plane count, slot q mod NS
                if (j > j1 || *abort_flag) break;
                const unsigned full = bar0 + 8 * s, empty = bar0 + 8 * (NS + s);
                if (q >= NS && !wide_wait(empty, (unsigned)((q / NS - 1) & 1), abort_flag)) break;
                // this lane's spans: records to copy (dst, first point, count)
                // and records to zero (two runs)
                unsigned vd = 0, zd = 0, zd2 = 0;
                int vp = 0, vn = 0, zn = 0, zn2 = 0;
                if (rowlane && j <= jl) {
                    const SRow rw = srows[j * WY + r];
                    int ua = max(clo, rw.xmin - xb), ub = min(chi, rw.xmax - xb + 1);
                    if (ua >= ub) ua = ub = clo;
                    const unsigned drow = s_u + (unsigned)((s * G::SLOT + r * WX) * G::REC);
                    vd = drow + ua * G::REC;
                    vp = rw.start + xb + ua;
                    vn = ub - ua;
                    // re-zero what held mesh points at the slot's last use
                    const int z1a = pa[s], z1b = ua == ub ? pa[s] : min(pb[s], ua);
                    const int z2a = ua == ub ? pa[s] : max(pa[s], ub), z2b = pb[s];
                    zd = drow + z1a * G::REC;
                    zn = max(0, z1b - z1a);
                    zd2 = drow + z2a * G::REC;
                    zn2 = max(0, z2b - z2a);
                    pa[s] = ua;
                    pb[s] = ub;
                } else if (baselane && j >= 4) {
                    // mesh columns of tile row br at plane j - 4: one run
                    const int2 e = orows[(j - 4) * TY + br];
                    const int ba = e.y ? __ffs(e.y) - 1 : 0, bb = e.y ? 32 - __clz(e.y) : 0;
                    vd = s_b + (unsigned)((s * G::NPTS + br * TX + ba) * G::REC);
                    vp = e.x + tx0 + ba;
                    vn = bb - ba;
                }
                const unsigned bytes = __reduce_add_sync(0xffffffffu, (unsigned)(vn + zn + zn2) * G::REC);
                if (lane == 0)
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full), "r"(bytes)
                                 : "memory");
                __syncwarp();
                // one copy per run: the records of the mesh points, then the two
                // zero runs (boxes wholly before point 0)
                if (vn > 0) wide_box(vd, (rowlane ? maps.u : maps.b) + (vn - 1), c0, vp, full);
                if (zn > 0) wide_box(zd, maps.u + (zn - 1), c0, kWideZeroPoint, full);
                if (zn2 > 0) wide_box(zd2, maps.u + (zn2 - 1), c0, kWideZeroPoint, full);
                // potential of the interior points (zero outside the mesh)
                for (int i = pw; i < G::NPTS / 32 && j <= jl; i += NPW) {
                    const int pt = lane + 32 * i, py = pt / TX, px = pt - py * TX;
                    const int2 e = orows[j * TY + py];
                    const bool ok = (e.y >> px) & 1;
                    if constexpr (CS)
                        cp_async_small<8>(s_v + (unsigned)((s * G::NPTS + pt) * 8),
                                          (const float2 *)a.Vc + (ok ? e.x + tx0 + px : 0), ok ? 8 : 0);
                    else
                        cp_async_small<4>(s_v + (unsigned)((s * G::NPTS + pt) * 4), a.V + (ok ? e.x + tx0 + px : 0),
                                          ok ? 4 : 0);
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full) : "memory");
                issued = q + 1;
            }
        }
        cp_async_wait<0>();
        // the copies issued for the last planes have landed before the block
        // can leave (the compute warps wait for them too, unless aborted)
        for (int q = max(0, issued - NS); q < issued; q++) {
            const unsigned full = bar0 + 8 * (q % NS);
            volatile int never = 0;
            wide_wait(full, (unsigned)((q / NS) & 1), &never);
        }
        if (pw == 0 && lane == 0 && *abort_flag && a.err != nullptr) atomicExch(a.err, 2);
        return;
    }

    // ---------------------------------------------------- compute warps
    const int cc = lane & 15, xh = lane >> 4;
    const int xl = 2 * (2 * (warp & 3) + xh);    // tile-local x of the thread's first column
    const int yl = 2 * (warp >> 2);              // tile-local y of its first row
    const int k = k0 + cc;
    const bool vok = k < ld;
    const int x0 = tx0 + xl, y0 = ty0 + yl;
    // planes (0-based j) where any of the warp's 4 x 2 columns holds a
    // point; the lanes share out the planes
    int jc0 = 1 << 30, jc1 = -1;
    const int xw = 4 * (warp & 3);
    for (int jj = lane; jj < np; jj += 32) {
        const int m = orows[jj * TY + yl].y | orows[jj * TY + yl + 1].y;
        if ((m >> xw) & 15) {
            jc0 = min(jc0, jj);
            jc1 = max(jc1, jj);
        }
    }
    jc0 = __reduce_min_sync(0xffffffffu, jc0);
    jc1 = __reduce_max_sync(0xffffffffu, jc1);
    float fxy[4];
#pragma unroll
    for (int pt = 0; pt < 4; pt++) fxy[pt] = a.f0 + a.fx * (float)(x0 + (pt & 1)) + a.fy * (float)(y0 + (pt >> 1));
    const float2 w1 = make_float2(a.w[1], a.w[1]), w2 = make_float2(a.w[2], a.w[2]);
    const float2 w3 = make_float2(a.w[3], a.w[3]), w4 = make_float2(a.w[4], a.w[4]);
    const float w0c = 3.0f * a.w[0], ai = a.ai, ar = a.ar;
    constexpr int RW = WX * NC;   // float2 entries per slot row
    const float2 *uwin = (const float2 *)gbase + ((4 + yl) * WX + xl) * NC + cc;
    const float2 *bwin = (const float2 *)(gbase + (s_b - s_u)) + (yl * TX + xl) * NC + cc;
    // staged diagonal of the thread's first point (float, or float2 with CS)
    const float *vwin = (const float *)(gbase + (s_v - s_u)) + (yl * TX + xl) * (VBY / 4);
    float2 *const out2 = (float2 *)a.out;

    // q[pt][e]: partial sums of the outputs at planes j - 4 + e (e = 0..7)
    // before plane j is added
    float2 q[4][8];
#pragma unroll
    for (int pt = 0; pt < 4; pt++)
#pragma unroll
        for (int kk = 0; kk < 8; kk++) q[pt][kk] = make_float2(0.f, 0.f);

    int sl = 0;
    unsigned par = 0;
#pragma unroll 1
    for (int j = j0; j <= j1; j++) {
        const unsigned full = bar0 + 8 * sl, empty = bar0 + 8 * (NS + sl);
        if (!wide_wait(full, par, abort_flag)) break;
        if (j >= jc0 && j <= jc1 + 4) {
            float2 s[4], cen[4];
            if (j <= jc1) {
                const float2 *pw = uwin + sl * G::SLOT * NC;
#define QW(r, kk) pw[(r) * RW + (kk) * NC]
#pragma unroll
                for (int r = 0; r < 2; r++) {
                    float2 W[10];
#pragma unroll
                    for (int kk = 0; kk < 10; kk++) W[kk] = QW(r, kk);
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
#undef QW
                const float fz = a.fz * (float)(zbase + j) + w0c;
                if constexpr (CS) {
                    // complex diagonal: staged v_theta e^{2i theta} plus the centre weight
                    const float2 *vc = (const float2 *)vwin + sl * G::NPTS;
#pragma unroll
                    for (int pt = 0; pt < 4; pt++) {
                        const float2 dv = vc[(pt >> 1) * TX + (pt & 1)];
                        const float dr = dv.x + fxy[pt] + fz;
                        s[pt].x = fmaf(-dv.y, cen[pt].y, fmaf(dr, cen[pt].x, s[pt].x));
                        s[pt].y = fmaf(dv.y, cen[pt].x, fmaf(dr, cen[pt].y, s[pt].y));
                    }
                } else {
                    const float *vv = vwin + sl * G::NPTS;
#pragma unroll
                    for (int pt = 0; pt < 4; pt++) {
                        // diagonal: staged V (zero outside the mesh) plus the field
                        const float d = vv[(pt >> 1) * TX + (pt & 1)] + fxy[pt] + fz;
                        s[pt].x = fmaf(d, cen[pt].x, s[pt].x);
                        s[pt].y = fmaf(d, cen[pt].y, s[pt].y);
                    }
                }
            } else {
#pragma unroll
                for (int pt = 0; pt < 4; pt++) s[pt] = cen[pt] = make_float2(0.f, 0.f);
            }
            // add plane j to the queues; the output of plane j - 4 completes
            float2 done[4];
#pragma unroll
            for (int pt = 0; pt < 4; pt++) {
                float2 *qq = q[pt];
                const float2 cv = cen[pt];
                done[pt] = f2_fma(w4, cv, qq[0]);
                qq[0] = f2_fma(w3, cv, qq[1]);
                qq[1] = f2_fma(w2, cv, qq[2]);
                qq[2] = f2_fma(w1, cv, qq[3]);
                qq[3] = f2_add(qq[4], s[pt]);
                qq[4] = f2_fma(w1, cv, qq[5]);
                qq[5] = f2_fma(w2, cv, qq[6]);
                qq[6] = f2_fma(w3, cv, qq[7]);
                qq[7] = f2_mul(w4, cv);
            }
            const int zo = zbase + j - 4;
            if (zo >= tl.zlo && zo < tl.zhi && vok) {
                const int2 *ro = orows + (j - 4) * TY + yl;
                const float2 *bb = bwin + sl * G::NPTS * NC;
#pragma unroll
                for (int dy = 0; dy < 2; dy++) {
                    const int2 e = ro[dy];
                    const int orow = (e.x + x0) * ld + k;
                    const int m = e.y >> xl;
#pragma unroll
                    for (int dx = 0; dx < 2; dx++) {
                        const float2 acc = done[2 * dy + dx];
                        const float2 bv = bb[(dy * TX + dx) * NC];
                        if constexpr (EPI == 1) {
                            const float2 y = make_float2(fmaf(-ai, acc.y, bv.x), fmaf(ai, acc.x, bv.y));
                            if ((m >> dx) & 1) out2[orow + dx * ld] = y;
                        } else if constexpr (EPI == 2) {
                            const float2 y = make_float2(fmaf(-ai, acc.y, fmaf(ar, acc.x, bv.x)),
                                                         fmaf(ai, acc.x, fmaf(ar, acc.y, bv.y)));
                            if ((m >> dx) & 1) out2[orow + dx * ld] = y;
                        } else {
                            if ((m >> dx) & 1) wide_finish(a, orow + dx * ld, acc, bv);
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty) : "memory");
        if (++sl == NS) {
            sl = 0;
            par ^= 1u;
        }
    }
}

// ------------------------------------------------------------- host side
typedef CUresult (*WideEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static WideEncodeFn wide_encode_fn() {
    static WideEncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (WideEncodeFn)p;
    });
    return fn;
}

// Boxes of 1 .. 24 records (16 complex64 values each) over the (P, ld)
// complex64 block at p, as (points, 2 ld floats); out-of-range rows read
// zero.  Encoded once per (pointer, ld, P) and kept.
static bool wide_maps_for(const void *p, int64_t P, int ld, CUtensorMap out[24]) {
    struct Key {
        const void *p;
        int64_t P;
        int ld;
        bool operator==(const Key &o) const { return p == o.p && P == o.P && ld == o.ld; }
    };
    struct KeyHash {
        size_t operator()(const Key &k) const {
            return std::hash<const void *>()(k.p) ^ (std::hash<int64_t>()(k.P) * 31u) ^ (size_t)k.ld * 1315423911u;
        }
    };
    static std::mutex mu;
    static std::unordered_map<Key, std::array<CUtensorMap, 24>, KeyHash> cache;
    std::lock_guard<std::mutex> lock(mu);
    const Key key{p, P, ld};
    auto it = cache.find(key);
    if (it == cache.end()) {
        WideEncodeFn fn = wide_encode_fn();
        if (!fn) return false;
        std::array<CUtensorMap, 24> m;
        for (int i = 0; i < 24; i++) {
            cuuint64_t dims[2] = {(cuuint64_t)2 * ld, (cuuint64_t)P};
            cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
            cuuint32_t box[2] = {32, (cuuint32_t)(i + 1)};
            cuuint32_t es[2] = {1, 1};
            if (fn(&m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(p), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        }
        if (cache.size() >= 256) cache.clear();
        it = cache.emplace(key, m).first;
    }
    for (int i = 0; i < 24; i++) out[i] = it->second[i];
    return true;
}

void wide_shape(const TileCfg &cfg, int *TX, int *TY) {
    *TX = 16;
    *TY = cfg.wty == 6 || cfg.wty == 4 ? cfg.wty : 8;
}

size_t wide_smem_bytes(int nyp, int ns, int zseg, int cs) {
    const size_t tx = 16, ty = 2 * (size_t)nyp, wx = tx + 8, wy = ty + 8;
    return 1024 + (size_t)ns * (wy * wx * 128 + tx * ty * 128 + tx * ty * (cs ? 8 : 4)) +
           (wy * sizeof(SRow) + ty * 8) * ((size_t)zseg + 8) + 8 + 16 * (size_t)ns + 16;
}

template <int NYP, int NS, int NPW, int CS = 0>
static cudaError_t launch_wide_t(const ApplyArgs<float> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                                 bool *launched) {
    // the Horner stage out = (-i tau / k) H u + psi has its own epilogue
    const bool horner = a.ar == 0.f && a.base != nullptr && a.br == 1.f && a.bi == 0.f && a.acc == nullptr;
    using G = WideGeom<NYP, NPW>;
    const size_t smem = wide_smem_bytes(NYP, NS, cfg.zseg, CS);
    if (smem > 227 * 1024) return cudaSuccess;
    const int ld = 2 * a.SV;
    WideMaps maps;
    if (!wide_maps_for(a.in, a.P, ld, maps.u)) return cudaSuccess;
    CUtensorMap bm[24];
    if (!wide_maps_for(a.base != nullptr ? a.base : a.in, a.P, ld, bm)) return cudaSuccess;
    for (int i = 0; i < 16; i++) maps.b[i] = bm[i];
    // complex scaling: alpha carries the rotation, so its Horner stage has a
    // complex alpha
    auto kern = k_apply_wide<NYP, NS, NPW, 0, CS>;
    if constexpr (CS == 0) {
        if (horner) kern = k_apply_wide<NYP, NS, NPW, 1, 0>;
    } else {
        if (a.base != nullptr && a.br == 1.f && a.bi == 0.f && a.acc == nullptr) kern = k_apply_wide<NYP, NS, NPW, 2, CS>;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nchunks = (ld + G::NC - 1) / G::NC;
    const long long nblk = (long long)ntiles * nchunks;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)nblk, G::NT, smem, st>>>(a, nchunks, maps);
    *launched = true;
    return cudaGetLastError();
}

cudaError_t launch_apply_wide(const ApplyArgs<float> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                              bool *launched) {
    *launched = false;
    // complex offsets are 32-bit; window coordinates are 16-bit
    if (ntiles == 0 || (long long)a.P * 2 * a.SV >= 0x7fffffffLL || a.nx > 32000) return cudaSuccess;
    // the tensor view needs 16-byte aligned blocks (ld is even for complex64)
    if (((uintptr_t)a.in & 15) != 0 || (a.base != nullptr && ((uintptr_t)a.base & 15) != 0)) return cudaSuccess;
    if (a.err == nullptr) return cudaSuccess;
    // complex scaling: the default shape only (6-row tiles, 4 producer
    // warps), no field
    if (a.Vc != nullptr) {
        if (cfg.wty != 6 || cfg.npw != 4 || ((uintptr_t)a.Vc & 7) != 0 || a.f0 != 0.f || a.fx != 0.f ||
            a.fy != 0.f || a.fz != 0.f)
            return cudaSuccess;
        return launch_wide_t<3, 3, 4, 1>(a, cfg, ntiles, st, launched);
    }
    // tile rows and slots: 8-row and 6-row tiles with 3 slots, 4-row tiles
    // with 4; 1 to 4 producer warps
#define RSG_WIDE_NPW(NYP_, NS_)                                                        \
    switch (cfg.npw) {                                                                 \
    case 1: return launch_wide_t<NYP_, NS_, 1>(a, cfg, ntiles, st, launched);          \
    case 2: return launch_wide_t<NYP_, NS_, 2>(a, cfg, ntiles, st, launched);          \
    case 3: return launch_wide_t<NYP_, NS_, 3>(a, cfg, ntiles, st, launched);          \
    default: return launch_wide_t<NYP_, NS_, 4>(a, cfg, ntiles, st, launched);         \
    }
    if (cfg.wty == 4) RSG_WIDE_NPW(2, 4)
    if (cfg.wty == 6) RSG_WIDE_NPW(3, 3)
    RSG_WIDE_NPW(4, 3)
#undef RSG_WIDE_NPW
}

}  // namespace rsg
