// Persistent batched time step for batches of complex64 systems.
//
// A batch is many independent systems, each a block of states on its own
// mesh with its own potential and projectors (arXiv:1501.05654, Sec.
// "Parallelization, optimizations and graphics processing units": a group of
// states is the unit of work; many small problems fill the device together).
// One launch of k_batch_step runs every Horner stage of one time step of
// every system: four stages per Taylor-4 exponential, out = psi + (-i tau/k)
// H u, eight for an ETRS step.
//
// Blocks stay resident (one per SM) and take work items from a queue, in
// queue order:
//   - dot:     the projector coefficients of one atom, c_i = h^3 <p_i|u>,
//              and D = h_a c (FP64 sums, one block per atom);
//   - stencil: one tile column segment of the local part (kinetic stencil,
//              potential, Horner epilogue), staged by producer warps;
//   - scatter: the projector terms of a run of points, out += (-i tau/k)
//              sum_a p_a D_a.
// The queue holds the items of stage t of every system before those of
// stage t + 1.  An item waits only for the items of its own system that
// produce what it reads or that read what it overwrites:
//   - dot and stencil of stage t: all items of stage t - 1;
//   - scatter of stage t: the dots and the stencil items of stage t.
// Every item waits only for items earlier in the queue, which blocks that
// are running already hold, so the waits end without any assumption about
// how many blocks are resident.  Each wait is bounded.  A wait that gives up
// sets a batch-wide abort flag and the status 2 (RSG_ERR_TIMEOUT); every
// block then leaves at its next item.
//
// The stencil item is the warp-specialised z-march of the single-system
// tensor-copy kernel, with the whole point record of the system (ld complex
// values, up to 16) as the staged unit.  A run of consecutive mesh points is
// then one contiguous piece of the state block and moves as one bulk copy;
// window positions outside the mesh are filled by bulk copies from a zero
// page.  The tile shape follows the record width, so that every block has
// the same 384 compute threads: one thread per complex value at two columns
// and two rows of the tile.  Systems with more than 16 values per point take
// 16-value chunks, one bulk copy per record.
#include "rsg_async.cuh"
#include "rsg_internal.h"
#include "rsg_vec.cuh"

namespace rsg {

namespace {

constexpr int kBNCW = 12;                    // compute warps
constexpr int kBNPW = 4;                     // producer warps
constexpr int kBNT = 32 * (kBNCW + kBNPW);   // threads per block
constexpr int kBNS = 3;                      // pipeline slots
constexpr unsigned kBSuspendNs = 2000;
constexpr long kBSlotWaitLimit = 1L << 20;   // about 2 s per slot wait

// Tile (TX x TY) of a system whose staged record holds LS complex values.
// Variant 0: one compute thread per value (LANES = LS) at two columns and two
// rows of the tile, wide rows where the record is short (fewer, longer
// copies).  Below 16 values the thread's two columns are x and x + TX / 2
// (not x and x + 1), so that the lanes of a warp read consecutive records:
// adjacent pairs would put the lanes two records apart and, with records
// shorter than 128 bytes, on the same shared-memory banks.  Variant 1
// (LS = 14), which the autotuner may choose: 16 value lanes (two idle) and
// adjacent columns on a 16 x 6 tile.
template <int LS, int VAR>
struct BTile;
template <> struct BTile<2, 0> { static constexpr int TX = 32, TY = 24, LANES = 2; };
template <> struct BTile<4, 0> { static constexpr int TX = 32, TY = 12, LANES = 4; };
template <> struct BTile<6, 0> { static constexpr int TX = 32, TY = 8, LANES = 6; };
template <> struct BTile<8, 0> { static constexpr int TX = 32, TY = 6, LANES = 8; };
template <> struct BTile<10, 0> { static constexpr int TX = 18, TY = 8, LANES = 10; };
template <> struct BTile<12, 0> { static constexpr int TX = 16, TY = 8, LANES = 12; };
template <> struct BTile<14, 0> { static constexpr int TX = 18, TY = 6, LANES = 14; };
template <> struct BTile<16, 0> { static constexpr int TX = 16, TY = 6, LANES = 16; };
template <> struct BTile<14, 1> { static constexpr int TX = 16, TY = 6, LANES = 16; };
// record lengths with variant 1
__host__ __device__ constexpr bool bhas_var1(int ls) { return ls == 14; }

// Staging geometry of records of LS complex values
template <int LS, int VAR>
struct BShape {
    static constexpr int TX = BTile<LS, VAR>::TX, TY = BTile<LS, VAR>::TY, LANES = BTile<LS, VAR>::LANES;
    static constexpr int WX = TX + 8, WY = TY + 8;
    static constexpr int REC = LS * 8;             // bytes per staged record
    static constexpr int UB = WX * WY * REC;       // input window of one plane
    static constexpr int BB = TX * TY * REC;       // base values of one plane
    static constexpr int VB = TX * TY * 4;         // potential of one plane
    static constexpr int GX = TX / 2;              // 2 x 2 groups per tile row
    static constexpr int NG = GX * (TY / 2);       // groups per tile
    static_assert(TX % 2 == 0 && TY % 2 == 0 && LANES >= LS, "2 x 2 groups, a lane per value");
    static_assert(LANES * NG <= 32 * kBNCW, "one compute thread per value lane and point group");
    static_assert(WY + TY <= 32 * kBNPW, "one producer lane per window row and per base row");
    static_assert(TX <= 32 && WY <= kBWinRowsMax && TY <= kBTileRowsMax, "table sizes");
    static_assert(WX * REC <= kBZeroBytes, "the zero page covers a window row");
};

constexpr int bslot_need(int ub, int bb, int vb) { return ub + bb + vb; }
static_assert(kBMaxLd % 2 == 0, "complex64 rows are whole float4");
constexpr int bmax(int a, int b) { return a > b ? a : b; }
template <int LS, int VAR>
constexpr int bslot_ls() { return bslot_need(BShape<LS, VAR>::UB, BShape<LS, VAR>::BB, BShape<LS, VAR>::VB); }
constexpr int kBSlot =
    (bmax(bmax(bmax(bmax(bslot_ls<2, 0>(), bslot_ls<4, 0>()), bmax(bslot_ls<6, 0>(), bslot_ls<8, 0>())),
               bmax(bmax(bslot_ls<10, 0>(), bslot_ls<12, 0>()), bmax(bslot_ls<14, 0>(), bslot_ls<16, 0>()))),
          bslot_ls<14, 1>()) +
     1023) & ~1023;
static_assert(9 * 4 * (kBNT + kBMaxLd / 2) * 8 <= kBNS * kBSlot, "the dot reduction fits in the ring");

// shared memory: ring of slots, window-row and tile-row tables, barriers,
// flags (block abort, current item)
struct BLayout {
    int off_srows, off_orows, off_bar, off_flag, bytes;
};
__host__ __device__ inline BLayout blayout(int np_cap) {
    BLayout L;
    L.off_srows = kBNS * kBSlot;
    L.off_orows = L.off_srows + kBWinRowsMax * np_cap * (int)sizeof(SRow);
    L.off_bar = L.off_orows + kBTileRowsMax * np_cap * (int)sizeof(int2);
    L.off_flag = L.off_bar + 16 * kBNS;
    L.bytes = L.off_flag + 32;
    return L;
}

__device__ __forceinline__ bool bs_wait(unsigned bar, unsigned parity, volatile int *abort_flag) {
    for (long it = 0; it < kBSlotWaitLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(kBSuspendNs)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// bulk copy of `bytes` (a multiple of 16) from global to shared memory,
// completing on the mbarrier
__device__ __forceinline__ void bs_copy(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait (thread 0) until *p >= need; false on the bound or a batch abort.
__device__ bool bs_dep_wait(const unsigned *p, unsigned need, long limit, const int *gabort) {
    for (long it = 0;; ++it) {
        if (ld_acquire(p) >= need) return true;
        if (it >= limit || *(volatile const int *)gabort) return false;
        __nanosleep(500);
    }
}

// ------------------------------------------------------------ stencil item
// The z-march over one tile column segment of one system (see the file
// comment).  Only planes [j0, j1] are staged: from the first plane with a
// point in the tile's own columns to four planes past the last one (jl);
// planes outside hold no value that reaches an output of the segment.  The
// last four carry only the base values of the outputs they complete.  J
// counts the planes the block staged before this item: slot and mbarrier
// phase of plane j are (J + j - j0) mod NS and (J + j - j0) / NS.  Returns
// the number of planes staged.
template <int LS, int VAR>
__device__ int bs_stencil(const BStepArgs &A, int it, unsigned s_ring, unsigned char *gring, unsigned J) {
    const BLayout L = blayout(A.np_cap);
    SRow *srows = (SRow *)(gring + L.off_srows);
    int2 *orows = (int2 *)(gring + L.off_orows);
    const unsigned bar0 = s_ring + (unsigned)L.off_bar;
    volatile int *babort = (volatile int *)(gring + L.off_flag);
    const BItem w = A.items[it];
    const SysArgs &S = A.sys[w.sys];
    const BStage bs = A.st[w.kind >> 2];
    using G = BShape<LS, VAR>;
    constexpr int TX = G::TX, TY = G::TY, WX = G::WX, WY = G::WY, REC = G::REC, LANES = G::LANES;
    static_assert(G::UB + G::BB + G::VB <= kBSlot, "a plane fits in its slot");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Tile tl = S.tiles[w.a];
    const int np = tl.zhi - tl.zlo + 8;
    const int ny = S.ny, nz = S.nz, ld = S.ld;
    const int k0 = 16 * w.b;   // first complex value of the chunk (ld > 16)
    const int tx0 = tl.tx * TX, ty0 = tl.ty * TY;
    const int xb = tx0 - 4, ybase = ty0 - 4, zbase = tl.zlo - 4;
#pragma unroll 4
    for (int i = tid; i < WY * np; i += kBNT) {
        const int zz = i / WY;
        const int yy = ybase + (i - zz * WY);
        const int zg = zbase + zz;
        SRow r{0, 1, 0};
        if (yy >= 0 && yy < ny && zg >= 0 && zg < nz) {
            const Row g = S.rows[zg * ny + yy];
            r.start = g.start - g.xmin;
            r.xmin = (int16_t)g.xmin;
            r.xmax = (int16_t)g.xmax;
        }
        srows[i] = r;
    }
#pragma unroll 4
    for (int i = tid; i < TY * np; i += kBNT) {
        const int zz = i / TY;
        const int yy = ty0 + (i - zz * TY);
        const int zg = zbase + zz;
        int2 e = make_int2(0, 0);
        if (yy < ny && zg >= 0 && zg < nz) {
            const Row g = S.rows[zg * ny + yy];
            const int lo = max(g.xmin - tx0, 0), hi = min(g.xmax - tx0, TX - 1);
            e.x = g.start - g.xmin;
            e.y = lo <= hi ? (int)(((2u << hi) - 1u) & ~((1u << lo) - 1u)) : 0;
        }
        orows[i] = e;
    }
    __syncthreads();
    // planes with a point in the tile's own columns (every warp computes the
    // same range)
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
    if (jl < 0) return 0;
    const int j0 = jf, j1 = min(np - 1, jl + 4);

    if (warp >= kBNCW) {
        // ------------------------------------------------ producer warps
        const int pw = warp - kBNCW;
        const int r = pw + kBNPW * lane;
        const bool rowlane = r < WY;
        const bool baselane = r >= WY && r < WY + TY;
        const int br = r - WY;
        const bool halo = r < 4 || r >= TY + 4;
        const int clo = halo ? 4 : 0, chi = halo ? 4 + TX : WX;
        const bool chunked = ld > 16;
        const unsigned cb = chunked ? (unsigned)min(16, ld - k0) * 8u : (unsigned)REC;
        const char *ug = (const char *)S.vec[bs.src];
        const char *bg = (const char *)S.vec[0];
        // the state blocks were written by other blocks of this launch with
        // ordinary stores; order those before this thread's bulk copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        int pa[kBNS], pb[kBNS];
#pragma unroll
        for (int s = 0; s < kBNS; s++) {
            pa[s] = clo;
            pb[s] = chi;
        }
        int issued = 0;
        for (int j = j0; j <= j1; j++) {
            if (*babort) break;
            const unsigned jg = J + (unsigned)(j - j0);
            const int s = (int)(jg % kBNS);
            const unsigned full = bar0 + 8 * s, empty = bar0 + 8 * (kBNS + s);
            if (jg >= (unsigned)kBNS && !bs_wait(empty, (jg / kBNS - 1u) & 1u, babort)) break;
            const unsigned slot = s_ring + (unsigned)(s * kBSlot);
            unsigned vd = 0, zd = 0, zd2 = 0;
            int vp = 0, vn = 0, zn = 0, zn2 = 0;
            int ps = s;
            if (rowlane && j <= jl) {
                const SRow rw = srows[j * WY + r];
                int ua = max(clo, rw.xmin - xb), ub = min(chi, rw.xmax - xb + 1);
                if (ua >= ub) ua = ub = clo;
                const unsigned drow = slot + (unsigned)(r * WX * REC);
                vd = drow + ua * REC;
                vp = rw.start + xb + ua;
                vn = ub - ua;
                // re-zero what held mesh points at the slot's last use
                int pas = pa[0], pbs = pb[0];
#pragma unroll
                for (int q = 1; q < kBNS; q++)
                    if (q == ps) {
                        pas = pa[q];
                        pbs = pb[q];
                    }
                const int z1a = pas, z1b = ua == ub ? pas : min(pbs, ua);
                const int z2a = ua == ub ? pas : max(pas, ub), z2b = pbs;
                zd = drow + z1a * REC;
                zn = max(0, z1b - z1a);
                zd2 = drow + z2a * REC;
                zn2 = max(0, z2b - z2a);
#pragma unroll
                for (int q = 0; q < kBNS; q++)
                    if (q == ps) {
                        pa[q] = ua;
                        pb[q] = ub;
                    }
            } else if (baselane && j >= 4) {
                const int2 e = orows[(j - 4) * TY + br];
                const int ba = e.y ? __ffs(e.y) - 1 : 0, bb = e.y ? 32 - __clz(e.y) : 0;
                vd = slot + (unsigned)(G::UB + (br * TX + ba) * REC);
                vp = e.x + tx0 + ba;
                vn = bb - ba;
            }
            const unsigned bytes =
                __reduce_add_sync(0xffffffffu, (unsigned)vn * cb + (unsigned)(zn + zn2) * (unsigned)REC);
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full), "r"(bytes)
                             : "memory");
            __syncwarp();
            const char *src = (rowlane ? ug : bg) + ((size_t)vp * ld + k0) * 8;
            if (!chunked) {
                if (vn > 0) bs_copy(vd, src, (unsigned)vn * REC, full);
            } else {
                for (int i = 0; i < vn; i++) bs_copy(vd + i * REC, src + (size_t)i * ld * 8, cb, full);
            }
            if (zn > 0) bs_copy(zd, A.zeros, (unsigned)(zn * REC), full);
            if (zn2 > 0) bs_copy(zd2, A.zeros, (unsigned)(zn2 * REC), full);
            // potential of the interior points (zero outside the mesh)
            for (int i = pw; i < (TX * TY + 31) / 32 && j <= jl; i += kBNPW) {
                const int pt = lane + 32 * i, py = pt / TX, px = pt - py * TX;
                if (pt < TX * TY) {
                    const int2 e = orows[j * TY + py];
                    const bool ok = (e.y >> px) & 1;
                    cp_async_small<4>(slot + (unsigned)(G::UB + G::BB + pt * 4), S.V + (ok ? e.x + tx0 + px : 0),
                                      ok ? 4 : 0);
                }
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full) : "memory");
            issued = j - j0 + 1;
        }
        cp_async_wait<0>();
        if (*babort) {
            // the copies issued for the last planes land before the block
            // moves on (the compute warps may have stopped waiting for them)
            for (int q = max(0, issued - kBNS); q < issued; q++) {
                const unsigned jg = J + (unsigned)q;
                volatile int never = 0;
                bs_wait(bar0 + 8 * (jg % kBNS), (jg / kBNS) & 1u, &never);
            }
        }
        return j1 - j0 + 1;
    }

    // ---------------------------------------------------- compute warps
    const int c = tid % LANES, g0 = tid / LANES;
    // threads past the tile's groups compute for the last group, lanes past
    // the record for its last value; neither stores
    const bool gok = g0 < G::NG;
    const int g = gok ? g0 : G::NG - 1;
    // the thread's points: columns xl and xl + XS, rows yl and yl + 1
    constexpr bool SPLIT = LANES == LS && LS < 16;
    constexpr int XS = SPLIT ? G::GX : 1;
    const int xl = SPLIT ? g % G::GX : 2 * (g % G::GX), yl = 2 * (g / G::GX);
    const int cc = c < LS ? c : LS - 1;
    const int k = k0 + c;
    const bool vok = gok && c < LS && k < ld;
    const int x0 = tx0 + xl;
    // planes where any of the thread's four points is a mesh point (first
    // and last, scanning from both ends), united over the warp
    int jc0 = np, jc1 = -1;
    {
        const unsigned need = (1u << xl) | (1u << (xl + XS));
        for (int jj = 0; jj < np; jj++)
            if ((unsigned)(orows[jj * TY + yl].y | orows[jj * TY + yl + 1].y) & need) {
                jc0 = jj;
                break;
            }
        for (int jj = np - 1; jj >= jc0; jj--)
            if ((unsigned)(orows[jj * TY + yl].y | orows[jj * TY + yl + 1].y) & need) {
                jc1 = jj;
                break;
            }
        if (jc1 < 0) jc0 = 1 << 30;
    }
    jc0 = __reduce_min_sync(0xffffffffu, jc0);
    jc1 = __reduce_max_sync(0xffffffffu, jc1);
    const float2 w1 = make_float2(S.w[1], S.w[1]), w2 = make_float2(S.w[2], S.w[2]);
    const float2 w3 = make_float2(S.w[3], S.w[3]), w4 = make_float2(S.w[4], S.w[4]);
    const float w0c = 3.0f * S.w[0], ai = bs.ai;
    constexpr int RW = WX * LS;   // float2 entries per window row
    const int uoff = ((4 + yl) * WX + xl) * LS + cc;
    const int boff = (G::UB / 8) + (yl * TX + xl) * LS + cc;
    const int voff = (G::UB + G::BB) / 4 + yl * TX + xl;
    float2 *const out2 = (float2 *)S.vec[bs.dst];

    float2 q[4][8];
#pragma unroll
    for (int pt = 0; pt < 4; pt++)
#pragma unroll
        for (int kk = 0; kk < 8; kk++) q[pt][kk] = make_float2(0.f, 0.f);

#pragma unroll 1
    for (int j = j0; j <= j1; j++) {
        const unsigned jg = J + (unsigned)(j - j0);
        const int sl = (int)(jg % kBNS);
        const unsigned full = bar0 + 8 * sl, empty = bar0 + 8 * (kBNS + sl);
        if (!bs_wait(full, (jg / kBNS) & 1u, babort)) break;
        if (j >= jc0 && j <= jc1 + 4) {
            const unsigned char *slotp = gring + (size_t)sl * kBSlot;
            float2 s[4], cen[4];
            if (j <= jc1) {
                const float2 *pw = (const float2 *)slotp + uoff;
#define QW(r, kk) pw[(r) * RW + (kk) * LS]
                if constexpr (SPLIT) {
                    // two 9-point x windows per row, TX / 2 apart
#pragma unroll
                    for (int r = 0; r < 2; r++) {
#pragma unroll
                        for (int dx = 0; dx < 2; dx++) {
                            float2 W[9];
#pragma unroll
                            for (int kk = 0; kk < 9; kk++) W[kk] = QW(r, kk + dx * XS);
                            cen[2 * r + dx] = W[4];
                            float2 t = f2_mul(w1, f2_add(W[3], W[5]));
                            t = f2_fma(w2, f2_add(W[2], W[6]), t);
                            t = f2_fma(w3, f2_add(W[1], W[7]), t);
                            s[2 * r + dx] = f2_fma(w4, f2_add(W[0], W[8]), t);
                        }
                    }
                } else {
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
                }
#pragma unroll
                for (int dx = 0; dx < 2; dx++) {
                    const int cx = 4 + dx * XS;   // window column of the thread's point dx
                    const float2 m4 = QW(-4, cx), m3 = QW(-3, cx), m2 = QW(-2, cx), m1 = QW(-1, cx);
                    const float2 p2 = QW(2, cx), p3 = QW(3, cx), p4 = QW(4, cx), p5 = QW(5, cx);
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
                const float *vv = (const float *)slotp + voff;
#pragma unroll
                for (int pt = 0; pt < 4; pt++) {
                    // diagonal: staged V (zero outside the mesh); no field
                    const float d = vv[(pt >> 1) * TX + (pt & 1) * XS] + w0c;
                    s[pt].x = fmaf(d, cen[pt].x, s[pt].x);
                    s[pt].y = fmaf(d, cen[pt].y, s[pt].y);
                }
            } else {
#pragma unroll
                for (int pt = 0; pt < 4; pt++) s[pt] = cen[pt] = make_float2(0.f, 0.f);
            }
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
                const float2 *bb = (const float2 *)slotp + boff;
#pragma unroll
                for (int dy = 0; dy < 2; dy++) {
                    const int2 e = ro[dy];
                    const int orow = (e.x + x0) * ld + k;
                    const int m = e.y >> xl;
#pragma unroll
                    for (int dx = 0; dx < 2; dx++) {
                        const float2 acc = done[2 * dy + dx];
                        const float2 bv = bb[(dy * TX + dx * XS) * LS];
                        const float2 y = make_float2(fmaf(-ai, acc.y, bv.x), fmaf(ai, acc.x, bv.y));
                        if ((m >> (dx * XS)) & 1) out2[orow + dx * XS * ld] = y;
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty) : "memory");
    }
    return j1 - j0 + 1;
}

// ---------------------------------------------------------------- dot item
// c_i = h^3 sum_q p_i(q) u(q) over the sphere entries of one atom, then
// D_i = sum_j h_a[i][j] c_j.  Thread (y, v): float4 v of the point row and
// entry lane y of ny = NT / SV; each lane sums its entries (every ny-th) in
// FP32, the lanes are summed in FP64: by warp shuffles and then over the
// warps when SV divides 32, else in lane order.  Shared memory (sm):
// the lane values (NP * 4 * NT doubles), the c values, and the atom's entry
// points when they fit.
template <int NP>
__device__ void bs_dot(const SysArgs &S, int atom, int src, unsigned char *sm) {
    using V = VT<float>;
    constexpr int UNR = NP > 4 ? 4 : 8;   // entries per lane and pass, loads in flight together
    const int tid = threadIdx.x, SV = S.SV;
    const int ny = kBNT / SV, y = tid / SV, v = tid - y * SV;
    double *red = (double *)sm;
    double *cv = red + NP * 4 * kBNT;
    int *qs = (int *)(cv + NP * 4 * kBMaxLd / 2);
    const int q0 = __ldg(S.chunk_q0 + __ldg(S.atom_chunk0 + atom));
    const int q1 = __ldg(S.chunk_q1 + __ldg(S.atom_chunk0 + atom + 1) - 1);
    const int nq = q1 - q0;
    const bool staged = (size_t)((unsigned char *)(qs + nq) - sm) <= (size_t)kBNS * kBSlot;
    if (staged) {
#pragma unroll 4
        for (int i = tid; i < nq; i += kBNT) qs[i] = __ldg(S.q_pt + q0 + i);
        __syncthreads();
    }
    const float4 *u = (const float4 *)S.vec[src];
    const float *qp = S.q_p + (size_t)q0 * NP;
    float4 acc[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) acc[i] = V::zero();
    if (y < ny) {
        int q = y;
        for (; q + (UNR - 1) * ny < nq; q += UNR * ny) {
            int pt[UNR];
#pragma unroll
            for (int k = 0; k < UNR; k++) pt[k] = staged ? qs[q + k * ny] : __ldg(S.q_pt + q0 + q + k * ny);
            float4 val[UNR];
#pragma unroll
            for (int k = 0; k < UNR; k++) val[k] = __ldcg(u + (size_t)pt[k] * SV + v);
#pragma unroll
            for (int k = 0; k < UNR; k++)
#pragma unroll
                for (int i = 0; i < NP; i++) V::fma(acc[i], __ldg(qp + (size_t)(q + k * ny) * NP + i), val[k]);
        }
        for (; q < nq; q += ny) {
            const int pt = staged ? qs[q] : __ldg(S.q_pt + q0 + q);
            const float4 val = __ldcg(u + (size_t)pt * SV + v);
#pragma unroll
            for (int i = 0; i < NP; i++) V::fma(acc[i], __ldg(qp + (size_t)q * NP + i), val);
        }
    }
    const int nval = NP * 4 * SV;
    if ((SV & (SV - 1)) == 0 && SV <= 32) {
        // SV divides 32: the lanes of a warp with the same v are SV apart;
        // warp shuffles sum them (a fixed tree), then the 16 warp sums of
        // each (i, comp, v) are added in warp order
        const int warp = tid >> 5, lane = tid & 31;
        constexpr int NW = kBNT / 32;
#pragma unroll
        for (int i = 0; i < NP; i++) {
            double d[4] = {acc[i].x, acc[i].y, acc[i].z, acc[i].w};
#pragma unroll
            for (int cmp = 0; cmp < 4; cmp++) {
                for (int off = SV; off < 32; off <<= 1) d[cmp] += __shfl_xor_sync(0xffffffffu, d[cmp], off);
                if (lane < SV) red[((i * 4 + cmp) * NW + warp) * SV + lane] = d[cmp];
            }
        }
        __syncthreads();
        for (int idx = tid; idx < nval; idx += kBNT) {
            const int ic = idx / SV, vv = idx - ic * SV;
            double sum = 0.0;
            for (int wq = 0; wq < NW; wq++) sum += red[(ic * NW + wq) * SV + vv];
            cv[idx] = S.h3 * sum;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NP; i++) {
            red[(i * 4 + 0) * kBNT + tid] = acc[i].x;
            red[(i * 4 + 1) * kBNT + tid] = acc[i].y;
            red[(i * 4 + 2) * kBNT + tid] = acc[i].z;
            red[(i * 4 + 3) * kBNT + tid] = acc[i].w;
        }
        __syncthreads();
        // (i, comp, v): the sum over the entry lanes in lane order, times
        // h^3, at cv[(i * 4 + comp) * SV + v]
        for (int idx = tid; idx < nval; idx += kBNT) {
            const int ic = idx / SV, vv = idx - ic * SV;
            const double *r = red + (size_t)ic * kBNT + vv;
            double sum = 0.0;
            for (int l = 0; l < ny; l++) sum += r[l * SV];
            cv[idx] = S.h3 * sum;
        }
    }
    __syncthreads();
    float *D = (float *)S.D;
    for (int idx = tid; idx < nval; idx += kBNT) {
        const int ic = idx / SV, vv = idx - ic * SV, i = ic >> 2, cmp = ic & 3;
        double dsum = 0.0;
        for (int jj = 0; jj < NP; jj++)
            dsum += __ldg(S.hm + ((size_t)atom * NP + i) * NP + jj) * cv[(jj * 4 + cmp) * SV + vv];
        D[(((size_t)atom * NP + i) * SV + vv) * 4 + cmp] = (float)dsum;
    }
}

// ------------------------------------------------------------ scatter item
// out += (-i tau/k) sum_a sum_i p_ai D_ai at cnt union points from u0.
// The item's point list, its entries (atom and projector values) and the
// system's D are first copied to shared memory with coalesced loads, when
// they fit; then thread (point lane, v), with NT / SV point lanes, takes
// four points per pass with their state loads in flight together.
constexpr int kBScD = 16384;     // bytes of D staged
constexpr int kBScEnt = 3072;    // entries staged
__device__ void bs_scatter(const SysArgs &S, int u0, int cnt, int dst, float ai, unsigned char *sm) {
    using V = VT<float>;
    const int tid = threadIdx.x, SV = S.SV, npmax = S.npmax;
    const int nD = S.natoms * npmax * SV;
    const int ea = __ldg(S.u_ptr + u0), ne = __ldg(S.u_ptr + u0 + cnt) - ea;
    float4 *dsm = (float4 *)sm;
    int *ipt = (int *)(sm + kBScD);
    int *iptr = ipt + kBScatterPts;
    int *iat = iptr + kBScatterPts + 1;
    float *ipv = (float *)(iat + kBScEnt);
    const bool dfit = nD * 16 <= kBScD, efit = ne <= kBScEnt;
    const float4 *Dg = (const float4 *)S.D;
    if (dfit)
#pragma unroll 4
        for (int i = tid; i < nD; i += kBNT) dsm[i] = __ldcg(Dg + i);
#pragma unroll 2
    for (int i = tid; i < cnt; i += kBNT) ipt[i] = __ldg(S.u_pts + u0 + i);
#pragma unroll 2
    for (int i = tid; i <= cnt; i += kBNT) iptr[i] = __ldg(S.u_ptr + u0 + i) - ea;
    if (efit) {
#pragma unroll 4
        for (int i = tid; i < ne; i += kBNT) iat[i] = __ldg(S.e_atom + ea + i);
#pragma unroll 4
        for (int i = tid; i < ne * npmax; i += kBNT) ipv[i] = __ldg(S.e_p + (size_t)ea * npmax + i);
    }
    __syncthreads();
    const float4 *D = dfit ? dsm : Dg;
    float4 *out = (float4 *)S.vec[dst];
    const int npt = kBNT / SV, pl = tid / SV, v = tid - pl * SV;
    if (pl >= npt) return;
    for (int b0 = pl; b0 < cnt; b0 += 4 * npt) {
        int pp[4];
        float4 o[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int i = b0 + k * npt;
            pp[k] = i < cnt ? ipt[i] : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) o[k] = pp[k] >= 0 ? __ldcg(out + (size_t)pp[k] * SV + v) : V::zero();
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (pp[k] < 0) continue;
            const int i = b0 + k * npt;
            float4 sum = V::zero();
            for (int e = iptr[i]; e < iptr[i + 1]; e++) {
                const int at = efit ? iat[e] : __ldg(S.e_atom + ea + e);
                const float *pv = efit ? ipv + (size_t)e * npmax : S.e_p + (size_t)(ea + e) * npmax;
                const float4 *Da = D + (size_t)at * npmax * SV + v;
                for (int j = 0; j < npmax; j++) V::fma(sum, pv[j], Da[(size_t)j * SV]);
            }
            out[(size_t)pp[k] * SV + v] = V::add(o[k], V::cmul(0.f, ai, sum));
        }
    }
}
static_assert(kBScD + (2 * kBScatterPts + 1 + kBScEnt) * 4 + kBScEnt * 9 * 4 <= kBNS * kBSlot,
              "the scatter item's tables fit in the ring");

__global__ void __launch_bounds__(kBNT, 1) k_batch_step(const __grid_constant__ BStepArgs A) {
    extern __shared__ __align__(128) unsigned char smraw[];
    const unsigned sraw = (unsigned)__cvta_generic_to_shared(smraw);
    const unsigned s_ring = (sraw + 1023u) & ~1023u;
    unsigned char *gring = smraw + (s_ring - sraw);
    const BLayout L = blayout(A.np_cap);
    const unsigned bar0 = s_ring + (unsigned)L.off_bar;
    volatile int *flags = (volatile int *)(gring + L.off_flag);   // [0] block abort, [1] item
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < kBNS; k++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * k), "r"(33 * kBNPW) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8 * (kBNS + k)), "r"(kBNCW)
                         : "memory");
        }
        flags[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned J = 0;   // planes staged by this block so far
    // thread 0 takes the next queue position while the block works on the
    // current item (a taken item is always worked on next, unless the batch
    // aborts)
    unsigned nxt = 0;
    if (tid == 0) nxt = atomicAdd(&A.ctl->head, 1u);
    for (;;) {
        if (tid == 0) {
            int it = -1;
            if (!*(volatile int *)&A.ctl->abort && nxt < (unsigned)A.nitems) it = (int)nxt;
            if (it >= 0) {
                nxt = atomicAdd(&A.ctl->head, 1u);
                const BItem w = A.items[it];
                const int stage = w.kind >> 2, kind = w.kind & 3;
                const SysArgs &S = A.sys[w.sys];
                const unsigned *cn = A.cnt + (size_t)w.sys * A.nst * 3;
                // (counter, count needed) pairs: stage t - 1 complete for dots and
                // stencil items, this stage's dots and stencil items for scatters
                const unsigned *cp = cn + (kind != 2 ? max(stage - 1, 0) : stage) * 3;
                const int nd = kind != 2 ? (stage > 0 ? 3 : 0) : 2;
                const unsigned need[3] = {(unsigned)S.ndot, (unsigned)(S.nsten + S.stall), (unsigned)S.nsca};
                bool ok = true;
                if (nd > 0) {
                    // all counters read at once; the bounded waits only when one is short
                    unsigned have[3];
#pragma unroll
                    for (int q = 0; q < 3; q++) have[q] = q < nd ? ld_acquire(cp + q) : 0u;
                    for (int q = 0; q < nd && ok; q++)
                        if (have[q] < need[q]) ok = bs_dep_wait(cp + q, need[q], A.wait_limit, &A.ctl->abort);
                }
                if (!ok) {
                    atomicExch(&A.ctl->abort, 1);
                    atomicExch(A.status, 2);
                    it = -1;
                }
            }
            flags[1] = it;
        }
        __syncthreads();
        const int it = flags[1];
        if (it < 0) break;
        const int kind0 = A.items[it].kind & 3;
        int staged = 0;
        if (kind0 == 1) {
            const SysArgs &S0 = A.sys[A.items[it].sys];
            const int ls = S0.ld > 16 ? 16 : S0.ld;
            const int var = S0.var == 1 && bhas_var1(ls) ? 1 : 0;
#define RSG_BS(L_, V_) staged = bs_stencil<L_, V_>(A, it, s_ring, gring, J)
            switch (ls * 4 + var) {
            case 8: RSG_BS(2, 0); break;
            case 16: RSG_BS(4, 0); break;
            case 24: RSG_BS(6, 0); break;
            case 32: RSG_BS(8, 0); break;
            case 40: RSG_BS(10, 0); break;
            case 48: RSG_BS(12, 0); break;
            case 56: RSG_BS(14, 0); break;
            case 57: RSG_BS(14, 1); break;
            default: RSG_BS(16, 0); break;
            }
#undef RSG_BS
        } else {
            const BItem w = A.items[it];
            const SysArgs &S = A.sys[w.sys];
            const BStage bs = A.st[w.kind >> 2];
            if (kind0 == 0) {
                switch (S.npmax) {
                case 1: bs_dot<1>(S, w.a, bs.src, gring); break;
                case 4: bs_dot<4>(S, w.a, bs.src, gring); break;
                default: bs_dot<9>(S, w.a, bs.src, gring); break;
                }
            } else {
                bs_scatter(S, w.a, w.b, bs.dst, bs.ai, gring);
            }
            // the ring is written by bulk copies again in later items
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        // this item's stores are read by later items, some through bulk copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
        const BItem w = A.items[it];
        if (tid == 0) {
            if (flags[0]) {
                atomicExch(&A.ctl->abort, 1);
                atomicExch(A.status, 2);
            } else {
                __threadfence();
                atomicAdd(A.cnt + ((size_t)w.sys * A.nst + (w.kind >> 2)) * 3 + (w.kind & 3), 1u);
            }
        }
        J += (unsigned)staged;
        if (flags[0]) break;
    }
}

}  // namespace

size_t batch_step_smem(int np_cap) { return 1024 + (size_t)blayout(np_cap).bytes; }

void batch_step_tile(int ld, int var, int *TX, int *TY) {
    const int ls = ld > 16 ? 16 : ld;
#define RSG_BT(L, V)              \
    *TX = BTile<L, V>::TX;        \
    *TY = BTile<L, V>::TY;        \
    return;
    if (var == 1 && bhas_var1(ls)) {
        RSG_BT(14, 1)
    }
    switch (ls) {
    case 2: RSG_BT(2, 0)
    case 4: RSG_BT(4, 0)
    case 6: RSG_BT(6, 0)
    case 8: RSG_BT(8, 0)
    case 10: RSG_BT(10, 0)
    case 12: RSG_BT(12, 0)
    case 14: RSG_BT(14, 0)
    default: RSG_BT(16, 0)
    }
#undef RSG_BT
}

int batch_step_threads() { return kBNT; }

cudaError_t launch_batch_step(const BStepArgs &a, int nblocks, cudaStream_t st) {
    const size_t smem = batch_step_smem(a.np_cap);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_step<<<nblocks, kBNT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rsg
