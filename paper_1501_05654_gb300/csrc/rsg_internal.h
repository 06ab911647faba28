// Internal declarations shared by the host API (rsg_host.cpp) and the CUDA
// kernels (rsg_kernels.cu, rsg_linalg.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rsg.h"

namespace rsg {

// One (y, z) row of the mesh bounding box: points x in [xmin, xmax] are
// stored contiguously from point index `start`.  Empty rows have xmin > xmax.
// Every supported shape (cube, box, sphere) meets each row in one interval.
struct Row {
    int32_t start, xmin, xmax, pad;
};

// Tile of the z-marching stencil kernel: bbox tile (tx, ty) and the planes
// [zlo, zhi) it produces.
struct Tile {
    int32_t tx, ty, zlo, zhi;
};

// Kernel tile configuration.
struct TileCfg {
    int kernel = 0;   // 0 shared-memory staged, 1 naive, 2 L1 z-march, 3 TMA gather, 4 row-TMA staged,
                      // 5 register-blocked staged (complex64), 7 warp-specialised tensor-copy staged (complex64)
    int rx = 1;       // points per thread along x
    int ty = 16;      // rows per tile (blockDim.z)
    int wty = 8;      // kernel 7: rows per tile, 8, 6 or 4
    int npw = 1;      // kernel 7: producer warps, 1 to 4
    int zseg = 120;   // planes per z segment
    int cv = 2;       // staged kernel: 16-byte vectors per point in a chunk (1..8)
    int stages = 4;   // staged kernels: shared-memory pipeline depth (3 or 4; kernel 4: 4 or 5 with 256 threads)
    int blocks_per_sm = 2;   // staged kernel, 256 threads: register budget for 2 or 3 blocks per SM
    int sync = 0;     // kernel 5, 192 threads: 0 block barrier per plane, 1/2 per-slot mbarriers
    int threads = 256;   // staged kernel: threads per block (256 with two blocks per SM, or 512)
};

// Everything one H application needs, by value.  Pointers to the state
// blocks are typed as the 16-byte vector of the compute type (float4 = two
// complex64 values, double2 = one complex128 value).
template <typename R>
struct ApplyArgs {
    const void *in;      // u (P, SV vectors)
    void *out;           // result
    const void *base;    // optional: added with scale beta
    void *acc;           // optional: acc = (acc_base or acc) + gamma * result
    const void *acc_base;    // optional: initial value of acc (acc is then write-only)
    const Row *rows;
    const Tile *tiles;
    int nx, ny, nz;
    int SV;              // 16-byte vectors per point row
    const R *V;          // local potential (P)
    R f0, fx, fy, fz;    // eps * dir.r = f0 + fx*ix + fy*iy + fz*iz (bbox idx)
    R w[5];              // -1/2 c_k / h^2
    R ar, ai, br, bi, gr, gi;
    // non-local part (may be absent: nl_ptr == nullptr)
    const int32_t *nl_ptr;   // P+1 CSR over points
    const int32_t *nl_ent;   // global sphere-entry index q
    const int32_t *q_atom;   // atom of each entry
    const R *q_p;            // entry-major projector values (npmax per entry)
    const void *D;           // (natoms*npmax, SV) vectors: h_a <p|u>
    int npmax;
    int64_t P;
    int *err;                // device status word (bounded waits record timeouts)
    // complex scaling in the register-blocked kernel: the complex diagonal
    // v_theta e^{2i theta} per point (interleaved); the caller folds the
    // kinetic rotation e^{-2i theta} into (ar, ai); nullptr otherwise
    const void *Vc = nullptr;
    // two-column blocks (ld = 2, one-thread-per-value kernels only): column c
    // has its own field terms cf[c] = (f0, fx, fy, fz) and alpha ca[c] =
    // (ar, ai) in place of (f0, fx, fy, fz) and (ar, ai); base and gamma are
    // shared
    int twocol = 0;
    R cf[2][4] = {};
    R ca[2][2] = {};
};

// Projector tables on the device (entry-major, see rsg_host.cpp).
struct ProjDev {
    int natoms = 0, npmax = 0;
    int64_t nq = 0;
    int nchunks = 0;
    int32_t *q_pt = nullptr;      // point of each entry
    int32_t *q_atom = nullptr;
    void *q_p = nullptr;          // R values, nq * npmax
    int32_t *chunk_atom = nullptr, *chunk_q0 = nullptr, *chunk_q1 = nullptr;
    int32_t *atom_chunk0 = nullptr; // natoms+1 prefix of chunks per atom
    double *hm = nullptr;         // natoms * npmax * npmax (zero padded)
    int32_t *nl_ptr = nullptr, *nl_ent = nullptr;
    int nu = 0;                    // points inside at least one sphere
    int32_t *u_pts = nullptr, *u_ptr = nullptr;   // those points and their CSR rows
    int32_t *e_atom = nullptr;     // per point-CSR entry: its atom (= q_atom[nl_ent[e]])
    void *e_p = nullptr;           // per point-CSR entry: its npmax projector values
};

// ---- launchers (rsg_kernels.cu) ----
// Block shape (cv x nxr x ty threads, tile TX = nxr * rx) of the staged kernel.
void stage_shape(const TileCfg &c, int SV, int *cv, int *nxr, int *ty);
// Block shape of the TMA-gather kernel (tile TX = nxr).
void tma_shape(const TileCfg &c, int SV, int *cv, int *nxr, int *ty);
// TMA-gather stencil (kernel 3); *launched = false when it does not apply.
template <typename R>
cudaError_t launch_apply_tma(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                             bool *launched);
// Register-blocked staged stencil (kernel 5, complex64): tile shape and
// launcher; *launched = false when it does not apply.
void quad_shape(const TileCfg &cfg, int *TX, int *TY);
cudaError_t launch_apply_quad(const ApplyArgs<float> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                              bool *launched);
// Warp-specialised stencil with tensor-copy staging (kernel 7, complex64,
// rsg_wide.cu): tile shape and launcher; *launched = false when it does not
// apply (unaligned blocks, complex scaling, shared memory too small).
void wide_shape(const TileCfg &cfg, int *TX, int *TY);
cudaError_t launch_apply_wide(const ApplyArgs<float> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                              bool *launched);
// Row-TMA staged stencil (kernel 4, the staged block shape); *launched =
// false when it does not apply.
template <typename R>
cudaError_t launch_apply_rowtma(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles, cudaStream_t st,
                                bool *launched);
template <typename R>
cudaError_t launch_apply(const ApplyArgs<R> &a, const TileCfg &cfg, int ntiles,
                         cudaStream_t st);
// Complex-scaled operator -1/2 e^{-2i theta} lap + v_theta (+ the real
// constant a.f0): vt holds the interleaved complex v_theta of every point;
// a.nl_ptr and the field terms are ignored (rsg_scaled.cu).
template <typename R>
cudaError_t launch_apply_scaled(const ApplyArgs<R> &a, const R *vt, double theta, cudaStream_t st);
// Coefficients D = h_a h^3 <p|u> in one launch: partial sums per chunk and
// the last block of each atom reducing them (counter: natoms * proj_slices
// zeroed words, left zeroed).
inline int proj_slices(int SV) {
    const int bv = SV < 32 ? SV : 32;   // vector slices of the coefficient kernels: bv vectors each
    return (SV + bv - 1) / bv;
}
template <typename R>
cudaError_t launch_proj_coeffs(const void *u, int SV, const ProjDev &pj, double *partial, unsigned *counter,
                               double h3, void *D, cudaStream_t st);
template <typename R>
cudaError_t launch_proj_dot(const void *u, int SV, const ProjDev &pj, double *partial,
                            cudaStream_t st);
template <typename R>
cudaError_t launch_proj_reduce(const double *partial, int SV, const ProjDev &pj,
                               double h3, void *D, cudaStream_t st);
// out += alpha * (projector terms), acc += gamma * alpha * (same), over the
// union points, reading the point-major entry copies (pj.e_atom, pj.e_p)
template <typename R>
cudaError_t launch_proj_scatter(const ApplyArgs<R> &a, const ProjDev &pj, cudaStream_t st);

// ---- linear algebra on state blocks (rsg_linalg.cu) ----
// G (S x S complex double) = h3 * Psi^H Phi (cross Gram; partial as launch_gram).
template <typename R>
cudaError_t launch_cross_gram(const void *psi, const void *phi, int64_t P, int ld, int S, double h3,
                              double *partial, int nblk, double *G, cudaStream_t st);
// psi <- psi Q (in place; Q S x S complex double).
template <typename R>
cudaError_t launch_rotate(void *psi, int64_t P, int ld, int S, const double *Q, cudaStream_t st);
// out[s] (complex double) = h3 sum_p x[p,s] y[p,s] (no conjugate; partial nblk * S * 2 doubles).
template <typename R>
cudaError_t launch_bilinear(const void *x, const void *y, int64_t P, int ld, int S, double h3, double *partial,
                            int nblk, double *out, cudaStream_t st);
// psi[p, s] *= M[p] (M: P values of the compute type), the first S states.
template <typename R>
cudaError_t launch_mask(void *psi, int64_t P, int ld, int S, const void *M, cudaStream_t st);
// z = a x + b y per state, complex a[s], b[s] (device, interleaved doubles); z may alias x or y.
template <typename R>
cudaError_t launch_comb(const void *x, const void *y, void *z, int64_t P, int ld, int S, const double *a,
                        const double *b, cudaStream_t st);
// out[s] = h3 sum_p |hx[p,s] - lam[s] x[p,s]|^2 (FP64; partial nblk * S doubles).
template <typename R>
cudaError_t launch_resid(const void *x, const void *hx, int64_t P, int ld, int S, const double *lam, double h3,
                         double *partial, int nblk, double *out, cudaStream_t st);
// G (S x S complex double) = h3 * Psi^H Psi; partial needs nblk * S * S * 2 doubles.
template <typename R>
cudaError_t launch_gram(const void *psi, int64_t P, int ld, int S, double h3,
                        double *partial, int nblk, double *G, cudaStream_t st);
int gram_blocks(int64_t P, int S);
// complex64 Gram: FP32 products in runs of 8 points, runs summed in FP64;
// the diagonal is replaced by the given FP64 norms (h3 applied).
cudaError_t launch_gram_c64(const void *psi, int64_t P, int ld, int S, double h3, double *partial,
                            int nblk, double *G, const double *norms, cudaStream_t st);
// complex64 triangular update with W^H rounded to FP32 (Wc_buf: S*S float2).
cudaError_t launch_tri_apply_c64(void *psi, int64_t P, int ld, int S, const double *W, void *Wc_buf,
                                 cudaStream_t st);
// In-place Cholesky of G, inverse of the factor into W (S x S complex double),
// drift[s] = max(drift[s], |G_ss - 1|), status word set non-zero on failure.
cudaError_t launch_chol_inv(double *G, double *W, int S, double *drift, int *status,
                            cudaStream_t st);
// psi <- psi W^H (in place).
template <typename R>
cudaError_t launch_tri_apply(void *psi, int64_t P, int ld, int S, const double *W,
                             cudaStream_t st);
// norms2[s] = h3 sum_p |psi[p,s]|^2 (FP64)
template <typename R>
cudaError_t launch_norms(const void *psi, int64_t P, int ld, int S, double h3,
                         double *partial, int nblk, double *out, cudaStream_t st);
int norm_blocks(int64_t P);
// Inner products for the adjoint: out[j*4+i] = h3 sum_p conj(b_j) x_p a_i for
// j + i <= 3 (complex double); b_j, a_i are P-vectors (S = 1, ld = 1 or 2).
template <typename R>
cudaError_t launch_adjoint_dots(const void *const *b, const void *const *a, int64_t P, int ld,
                                const R *X, double h3, double *partial, int nblk,
                                double *out, cudaStream_t st);
// Fused adjoint inner products + reduction + grad_k update (one launch);
// counter (device, zero on entry) is reset by the kernel.
template <typename R>
cudaError_t launch_adjoint_grad(const void *const *b, const void *const *a, int64_t P, int ld,
                                const R *X, double h3, double tau, double *partial, int nblk,
                                unsigned *counter, double *grad_k, cudaStream_t st);
// overlap: out = h3 sum_p conj(f_p) g_p  (complex double, one state)
template <typename R>
cudaError_t launch_overlap(const void *f, const void *g, int64_t P, int ld, double h3,
                           double *partial, int nblk, double *out, cudaStream_t st);
// y = a * x (+ y if accumulate), complex scalar a given as device double[2]
// or host values; one state vector or a whole block (n complex values).
template <typename R>
cudaError_t launch_axpby(const void *x, void *y, int64_t n, double ar, double ai,
                         double br, double bi, cudaStream_t st);
// y = x * (a[0] + i a[1]) where a is a DEVICE complex double (graph friendly)
template <typename R>
cudaError_t launch_scale_dev(const void *x, void *y, int64_t n, const double *a,
                             cudaStream_t st);
// grad[k] += 2 Re( -i tau * sum_n 1/n! sum_j M[j][n-1-j] )  (device)
cudaError_t launch_grad_accum(const double *M, double tau, double *grad_k,
                              cudaStream_t st);

// ---- batches of independent complex64 systems (rsg_kernels.cu) ----
// Per-system arguments, resident on the device.  vec[] = {psi, w0, w1}: the
// caller's state block and two work blocks; kernels pick input, output and
// base by index so one captured step serves every system.
struct SysArgs {
    void *vec[3];
    const Row *rows;
    const Tile *tiles;
    int nx, ny, nz, SV, P;
    const float *V;
    float w[5];
    int natoms, npmax, nu;
    const int32_t *q_pt, *q_atom, *nl_ent, *chunk_q0, *chunk_q1, *atom_chunk0, *u_pts, *u_ptr, *e_atom;
    const float *q_p, *e_p;
    const double *hm;
    float *D;
    double *partial;
    double h3;
    // persistent step (k_batch_step): complex values per point, and per
    // stage the number of dot (one per atom), stencil and scatter items;
    // stall > 0 makes the stencil count unreachable (a test of the bounded
    // waits)
    int ld, ndot, nsten, nsca, stall;
    int var;   // tile variant of the system's record length (0 or 1)
};
// Work item: stencil (sys, tile, chunk); projector dot (sys, chunk);
// projector reduce (sys, atom); scatter (sys, first union point).
struct BWork {
    int32_t sys, a, b, pad;
};
// Register-blocked stencil over every system's tiles (16 x 12 tiles, chunks
// of four complex values = two 16-byte vectors; rsg_quad.cu).
cudaError_t launch_batch_stencil(const SysArgs *sys, const BWork *work, int nwork, int in_c, int out_c,
                                 float ar, float ai, cudaStream_t st);
constexpr int kBatchCV = 2, kBatchTY = 12, kBatchNXR = 16, kBatchZseg = 120;
cudaError_t launch_batch_proj(const SysArgs *sys, const BWork *dot_work, int ndot, const BWork *red_work,
                              int nred, int in_c, int npmax, cudaStream_t st);
cudaError_t launch_batch_scatter(const SysArgs *sys, const BWork *work, int nwork, int out_c, float ar,
                                 float ai, cudaStream_t st);

// ---- persistent batched time step (rsg_bstep.cu) ----
// Stage t of a step: out = vec[dst] = psi + i ai H vec[src] (ai = -tau / k).
struct BStage {
    int src, dst;
    float ai;
};
// Work item: kind = 4 * stage + {0 dot (a = atom), 1 stencil (a = tile, b =
// 16-value chunk), 2 scatter (a = first union point, b = count)}.
struct BItem {
    int32_t kind, sys, a, b;
};
struct BCtl {
    unsigned head;   // next queue position
    int abort;       // set by a wait that gave up
};
constexpr int kBWinRowsMax = 32, kBTileRowsMax = 24;   // window and tile rows of any batch tile
constexpr int kBZeroBytes = 4096;                      // zero page read by the window fills
constexpr int kBScatterPts = 2048;                     // union points per scatter item
constexpr int kBMaxLd = 128;                           // complex values per point in the persistent step
struct BStepArgs {
    const SysArgs *sys;
    const BItem *items;
    int nitems, nst;
    BStage st[8];
    unsigned *cnt;       // (system, stage, kind): items finished
    BCtl *ctl;
    int *status;         // 2 when a bounded wait gave up
    const void *zeros;   // kBZeroBytes of zeros, 16-byte aligned
    long wait_limit;     // polls of a dependency wait (about 0.5 us each)
    int np_cap;          // planes of the longest tile segment plus 8
};
// Tile of a system with ld complex values per point (ld > 16: 16-value
// chunks) in tile variant var (0 or 1; the same tile where a record length
// has one variant).
void batch_step_tile(int ld, int var, int *TX, int *TY);
size_t batch_step_smem(int np_cap);
int batch_step_threads();
cudaError_t launch_batch_step(const BStepArgs &a, int nblocks, cudaStream_t st);

// Host-side accessors for code outside rsg_host.cpp: the Hamiltonian's
// compute type, point count and spacing, and the thread-local error message.
void ham_info(rsg_ham H, rsg_dtype *dtype, int64_t *P, double *spacing);
rsg_status set_error(rsg_status s, const char *msg);

}  // namespace rsg
