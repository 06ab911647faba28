/*
 * rsg.h -- C ABI of the real-space-grid Hamiltonian library (GB300, sm_103a).
 *
 * The library applies H = -1/2 lap + V_loc + eps(t) dir.r
 *                       + sum_a sum_ij |p_ai> h_a,ij <p_aj|
 * to a block of complex states sampled on a uniform real-space mesh, and
 * propagates the block in real time with a Taylor-4 exponential.  Sources
 * (arXiv:1501.05654):
 *   - Sec. 1: fields on uniform grids, integrals as grid sums, high-order
 *     finite-difference Laplacian; finite boxes of arbitrary shape.
 *   - Sec. "Parallelization, optimizations and graphics processing units": the building blocks include "the application of a
 *     Hamiltonian"; the basic object is a group of several states; a field is
 *     a linear array plus tables describing the grid; the point order in
 *     memory is the library's business.
 *   - Sec. "Magnetic response and gauge invariance in real-space grids": pseudopotentials act as a non-local operator
 *     (here separable projectors |p_ai> h_ij <p_aj|).
 *   - Sec. "Quantum optimal control", Eq. (qoctgradient): gradient of a
 *     final-time objective with respect to the control, through a costate
 *     propagated backwards with the same propagators.
 *
 * Conventions shared by every call:
 *   - All calls return an rsg_status; rsg_last_error() gives a thread-local
 *     message for the last failure.  No exception crosses the ABI.
 *   - Handles are owned by the library; destroy them with the matching call.
 *     The caller owns every state, potential, field and gradient buffer.
 *   - State blocks are DEVICE pointers to a row-major (P, ld) array of
 *     complex values, states fastest: element (p, s) at offset p*ld + s.
 *     complex64 = interleaved float pairs, complex128 = double pairs.  For
 *     complex64, ld must be even and the pointer 16-byte aligned; columns
 *     S..ld-1 are padding (computed on but never reduced over).
 *   - Points are in the LIBRARY's order (z slowest, then y, x fastest, over
 *     the mesh only).  rsg_mesh_coords gives each point's lattice integers.
 *     Position of lattice (i,j,k) = origin + spacing * (i,j,k).
 *   - Inner products are <f|g> = h^3 sum_p conj(f_p) g_p.
 *   - Calls taking `stream` (a cudaStream_t, NULL = legacy default stream)
 *     only enqueue work, unless they return host values (noted per call),
 *     which synchronises that stream.
 */
#ifndef RSG_H
#define RSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsg_mesh_s *rsg_mesh;
typedef struct rsg_ham_s *rsg_ham;
typedef struct rsg_batch_s *rsg_batch;

typedef enum {
    RSG_OK = 0,
    RSG_ERR_ARG = -1,          /* invalid argument (NULL, size, alignment) */
    RSG_ERR_OOM = -2,          /* device or host allocation failed */
    RSG_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    RSG_ERR_UNSUPPORTED = -4,  /* valid request the library does not support */
    RSG_ERR_TIMEOUT = -5,      /* a bounded device wait gave up (reported by the
                                  next call that synchronises the stream) */
    RSG_ERR_NONFINITE = -6,    /* a norm or Gram check found NaN/Inf */
    RSG_ERR_STATE = -7         /* handle not ready (e.g. missing potential) */
} rsg_status;

typedef enum { RSG_C64 = 0, RSG_C128 = 1 } rsg_dtype;
typedef enum { RSG_SHAPE_CUBE = 0, RSG_SHAPE_SPHERE = 1, RSG_SHAPE_BOX = 2 } rsg_shape;
typedef enum { RSG_EXPMID = 0, RSG_ETRS = 1 } rsg_scheme;
/* Boundary rule of the Laplacian: zero values outside the mesh (finite
 * systems, the default), or antisymmetric images for a cube or box. */
typedef enum { RSG_BC_ZERO = 0, RSG_BC_ODD = 1 } rsg_bc;

/* ---------------------------------------------------------------- mesh ---
 * Uniform mesh (Sec. 1; Sec. "Parallelization, optimizations and graphics processing units": field = linear array + grid
 * tables).  CUBE: n[0]^3 points, lattice i = 0..n-1, origin -(n-1)h/2 per
 * axis (centred box).  BOX: n[0] x n[1] x n[2], same centring.  SPHERE:
 * lattice points with i^2+j^2+k^2 <= (radius/spacing)^2 (inclusive,
 * rounded to 1e-6), origin 0.  Values outside the mesh are zero (the
 * Dirichlet boundary of the finite-system runs).  n is ignored for SPHERE
 * and radius for CUBE/BOX.  Every extent must be <= 1024 lattice points.
 * Errors: RSG_ERR_ARG for spacing <= 0, extents outside 1..1024, NULL out. */
rsg_status rsg_mesh_create(rsg_shape shape, const int32_t n[3], double radius,
                           double spacing, rsg_mesh *out);

/* Boundary rule of a cube or box mesh (Sec. 1: finite boxes; the image
 * rule is a test aid).  RSG_BC_ZERO (default): neighbours outside the mesh
 * are zero.  RSG_BC_ODD: a neighbour outside the mesh takes the value of
 * its mirror image about a wall one spacing outside the mesh, with the sign
 * flipped, and a neighbour on a wall is zero; minus the Laplacian then has
 * the closed-form eigenvalues sum_d sigma(pi m_d / (n_d + 1)) / h^2 with
 * products of sines as eigenvectors, so box eigenvalues converge at the
 * stencil's order.  Applications on an image-wall mesh run the
 * one-thread-per-value kernels (1, or 6 with complex scaling); batches
 * refuse such meshes.  Set it before building Hamiltonians' work on the
 * mesh or between calls (not while a call on the mesh is in flight).
 * A neighbour is reflected once, which reaches its image inside the mesh
 * only with at least 4 points along every axis.
 * Errors: RSG_ERR_ARG for an unknown rule or RSG_BC_ODD with an extent below
 * 4, RSG_ERR_UNSUPPORTED for RSG_BC_ODD on a sphere. */
rsg_status rsg_mesh_set_boundary(rsg_mesh m, int bc);
/* Number of mesh points P. */
rsg_status rsg_mesh_num_points(rsg_mesh m, int64_t *P);
/* Host array ijk (P x 3 int32, caller-owned): lattice integers of every point
 * in library order. */
rsg_status rsg_mesh_coords(rsg_mesh m, int32_t *ijk);
/* Position of lattice (0,0,0) and the spacing. */
rsg_status rsg_mesh_geometry(rsg_mesh m, double origin[3], double *spacing);
rsg_status rsg_mesh_destroy(rsg_mesh m);

/* ---------------------------------------------------------- Hamiltonian ---
 * A Hamiltonian bound to a mesh and a compute type.  complex64 computes the
 * stencil, potential and Taylor terms in FP32 and keeps FP64 for projector
 * coefficient reductions, norms and Gram matrices; complex128 is FP64
 * throughout.  The mesh must outlive the Hamiltonian. */
rsg_status rsg_ham_create(rsg_mesh m, rsg_dtype dtype, rsg_ham *out);
rsg_status rsg_ham_destroy(rsg_ham H);

/* Local potential V (P doubles, library point order).  v_on_device = 0:
 * host array; 1: device array.  Copied; the caller keeps ownership. */
rsg_status rsg_potential_set(rsg_ham H, const double *v, int v_on_device);

/* Separable projectors (Sec. "Magnetic response and gauge invariance in real-space grids": non-local pseudopotential).
 * Atom a at centres[3a..3a+2] (bohr) carries (lmax[a]+1)^2 projectors,
 * lmax in {0,1,2}: p_ai(r) = Y_i(r-R_a) exp(-|r-R_a|^2/(2 beta_a^2)) on the
 * mesh points with |r-R_a| <= rcut[a], Y = {1; x,y,z; xy,yz,zx,x^2-y^2,
 * 3z^2-r^2}, each scaled so that h^3 sum_p p_ai(p)^2 = 1.  hmats holds the
 * per-atom nproj x nproj coupling matrices h_a (row-major, concatenated,
 * symmetric).  natoms = 0 removes all projectors.  Host arrays, copied. */
rsg_status rsg_projectors_set(rsg_ham H, int natoms, const double *centres,
                              const double *rcut, const int32_t *lmax,
                              const double *beta, const double *hmats);

/* Separable projectors given as values (the same non-local term,
 * sum_a sum_ij |p_ai> h_a,ij <p_aj|, for projectors the caller samples
 * itself, e.g. from a pseudopotential table).  Atom a covers npts[a] mesh
 * points: point_idx (concatenated over atoms, library point order, each
 * point at most once per atom) and, for each of them in the same order,
 * nproj[a] values (pvals, concatenated, point-major: value i of the k-th
 * point of atom a at offset_a + k * nproj[a] + i).  The values are used as
 * given (no normalisation); hmats as in rsg_projectors_set (nproj x nproj
 * per atom, symmetric to 1e-12 of its largest entry).  Host arrays, copied;
 * replaces any projector set; natoms = 0 removes all projectors.
 * Errors: RSG_ERR_ARG for a NULL array, nproj < 1, npts < 0, a point index
 * outside the mesh or repeated within an atom, a non-finite value or an
 * asymmetric h; RSG_ERR_UNSUPPORTED for nproj > 9 or while complex scaling
 * is set. */
rsg_status rsg_projectors_set_raw(rsg_ham H, int natoms, const int64_t *npts, const int64_t *point_idx,
                                  const int32_t *nproj, const double *pvals, const double *hmats);

/* Static dipole field eps * (dir . r) used by rsg_hamiltonian_apply and
 * rsg_taylor_apply (default 0).  dir may be NULL when eps = 0. */
rsg_status rsg_field_set(rsg_ham H, double eps, const double dir[3]);

/* hpsi = H psi for S states (Sec. "Parallelization, optimizations and graphics processing units": application of a
 * Hamiltonian to a group of states).  psi and hpsi: device (P, ld) blocks of
 * the Hamiltonian's dtype; they must not overlap.  Asynchronous on stream.
 * Errors: RSG_ERR_ARG (NULL, S < 1, ld < S, odd ld for complex64, misaligned
 * pointer, overlap), RSG_ERR_STATE (no potential set). */
rsg_status rsg_hamiltonian_apply(rsg_ham H, const void *psi, void *hpsi, int64_t S,
                                 int64_t ld, void *stream);

/* out = T(tau) psi = sum_{n=0..4} (-i tau H)^n / n! psi (one Taylor-4
 * exponential of the real-time propagator, Sec. 2 real-time TDDFT).  out may
 * equal psi (in place).  Asynchronous. */
rsg_status rsg_taylor_apply(rsg_ham H, const void *psi, void *out, int64_t S,
                            int64_t ld, double tau, void *stream);

/* Propagates psi in place over nsteps intervals of length dt.  The field is
 * piecewise constant: eps[k] (host array, may be NULL = 0) on interval k,
 * along dir (NULL = x).  EXPMID: nsub exponentials T(dt/nsub) with
 * H(t_k + dt/2) per interval; ETRS: nsub pairs T_{H(t+dt')}(dt'/2)
 * T_{H(t)}(dt'/2), dt' = dt/nsub.  Every gs_every steps (0 = never) the
 * squared-norm drift |<psi_s|psi_s> - 1| is recorded (FP64) and the block is
 * re-orthonormalised by Cholesky-QR in FP64 (equal to Gram-Schmidt in index
 * order); the final block is checked too.  norm_drift_out (host, S doubles,
 * may be NULL) receives the largest drift seen per state, and synchronises.
 * Errors: as rsg_hamiltonian_apply; RSG_ERR_NONFINITE if a Gram matrix is not
 * finite or not positive definite. */
rsg_status rsg_propagate_steps(rsg_ham H, void *psi, int64_t S, int64_t ld,
                               int64_t nsteps, double dt, rsg_scheme scheme,
                               int nsub, const double *eps, const double dir[3],
                               int gs_every, double *norm_drift_out, void *stream);

/* Re-orthonormalises S states in place (Cholesky-QR, FP64 Gram and factor);
 * norms2_out (host, S, may be NULL) receives <psi_s|psi_s> before, and
 * synchronises. */
rsg_status rsg_orthonormalize(rsg_ham H, void *psi, int64_t S, int64_t ld,
                              double *norms2_out, void *stream);

/* Lowest S eigenpairs of H (the ground-state step before a propagation: the
 * paper's closing section on parallelisation names orthogonalisation and
 * subspace diagonalisation as the ground-state building blocks, and its
 * few-electron section tabulates the 1-D lithium eigenvalues this solves
 * for as one particle in 3-D).  Chebyshev-filtered subspace iteration: each
 * of max_iter iterations applies a degree-`degree` Chebyshev polynomial of H
 * (degree applications of H - c, damping the spectrum above the largest
 * current Ritz value), re-orthonormalises (FP64 Cholesky-QR) and does a
 * Rayleigh-Ritz step on the FP64 S x S matrix X^H H X.  It stops when the
 * residuals |H x_s - lambda_s x_s| (h^3-weighted 2-norm, FP64) of the nwant
 * lowest states are <= tol.  The S - nwant states above them are a buffer:
 * the filter damps the spectrum above the largest Ritz value, so wanted
 * states converge at a rate set by their distance from the buffer's top
 * (a few buffer states past the next gap in the spectrum are enough).
 * psi (device, P x ld, S <= 256): in, the starting block (any full-rank
 * block, e.g. seeded random values); out, the orthonormal Ritz vectors in
 * ascending order.  evals_out (host, S) receives the Ritz values, resid_out
 * (host, S, may be NULL) the residual norms, iters_out (may be NULL) the
 * iterations taken.  The current field (rsg_field_set) is part of H.
 * Uses the Hamiltonian's work blocks; synchronises once per iteration.
 * Errors: as rsg_hamiltonian_apply; RSG_ERR_ARG for degree outside 1..64,
 * nwant outside 1..S, max_iter < 0 or tol <= 0; RSG_ERR_UNSUPPORTED for S > 256;
 * RSG_ERR_NONFINITE if the block loses rank or a matrix is not finite. */
rsg_status rsg_eigensolve(rsg_ham H, void *psi, int64_t S, int64_t ld, int64_t nwant, int64_t max_iter,
                          int degree, double tol, double *evals_out, double *resid_out, int64_t *iters_out,
                          void *stream);

/* Mask absorber (Sec. "Photoemission", Eq. (mask_split): an orbital splits
 * into a bounded part M(r) phi and an unbounded part (1 - M(r)) phi; keeping
 * the bounded part removes the charge that reaches the boundary region).
 * mask: P values in [0, 1] in library point order (host, or device when
 * mask_on_device != 0); after every time step of rsg_propagate_steps each
 * state is multiplied by it pointwise.  NULL removes the absorber.  With an
 * absorber set, rsg_control_gradient and rsg_control_optimize (whose adjoint
 * is that of the propagator without it) and rsg_batch_create return
 * RSG_ERR_UNSUPPORTED.  Errors: RSG_ERR_ARG for a value outside [0, 1]. */
rsg_status rsg_absorber_set(rsg_ham H, const double *mask, int mask_on_device);

/* Complex scaling (Sec. "Complex scaling and resonances": the transform
 * R_theta maps H to H_theta, and the single-particle equation there takes
 * the kinetic term times e^{-2i theta} and the potential at the rotated
 * coordinates).  While set, every Hamiltonian application uses
 *   H_theta = -1/2 e^{-2i theta} lap + v_theta(r),
 * which is complex symmetric, not Hermitian: bound-state energies stay on
 * the real axis, the continuum turns by -2 theta, resonances appear as
 * eigenvalues eps0 - i Gamma/2.  v_theta: 2P doubles, the values
 * v(r e^{i theta}) of every point as (re, im) pairs in library point order
 * (host, or device when v_on_device != 0), computed by the caller, who
 * knows v analytically; copied, and used in place of rsg_potential_set's
 * V (which may be left unset).  theta in [0, pi/4].  v_theta = NULL
 * removes the scaling.  rsg_hamiltonian_apply, rsg_taylor_apply,
 * rsg_propagate_steps (without a field) and rsg_shifted_solve use H_theta;
 * rsg_eigensolve, rsg_control_gradient, rsg_control_optimize and
 * rsg_batch_create return RSG_ERR_UNSUPPORTED, as do rsg_projectors_set
 * with atoms and rsg_field_set or rsg_propagate_steps with a nonzero field
 * (and this call, while either is set).  complex64 applications with the
 * default kernel run the register-blocked stencil (kernel 5) with the
 * complex diagonal v_theta e^{2i theta} and e^{-2i theta} folded into the
 * output scaling; otherwise they run kernel 6 (one thread per point and
 * 16-byte vector).
 * Errors: RSG_ERR_ARG for theta outside [0, pi/4] or a non-finite value. */
rsg_status rsg_complex_scaling_set(rsg_ham H, double theta, const double *v_theta, int v_on_device);

/* Shifted linear solves (H - z) x = b for S right-hand sides at one complex
 * shift z = zr + i zi: the linear problem of the Sternheimer equation
 * (Sec. "The Sternheimer formulation of linear-response": a shifted
 * Kohn-Sham Hamiltonian is inverted at every step; a complex shift needs a
 * non-Hermitian solver).  Conjugate-orthogonal conjugate gradients for the
 * complex symmetric H - z (H is real symmetric: real stencil, potential,
 * field and projector matrices; or the complex-symmetric H_theta of
 * rsg_complex_scaling_set), each right-hand side its own system; A x
 * is one Hamiltonian application with -z x added in the epilogue; inner
 * products are FP64.  b (device, P x ld, read only); x (device, same
 * shape): in, the initial guess (zeros for none); out, the solution.  Stops
 * when every |b_s - (H - z) x_s| <= tol |b_s| or after max_iter iterations;
 * resid_out (host, S, may be NULL) receives the true relative residuals,
 * iters_out (may be NULL) the iterations.  Uses three work blocks of the
 * Hamiltonian; synchronises twice per iteration.
 * Errors: as rsg_hamiltonian_apply; RSG_ERR_ARG for overlapping b and x,
 * max_iter < 0, tol <= 0 or a non-finite shift; RSG_ERR_NONFINITE on a
 * breakdown (p^T (H - z) p = 0). */
rsg_status rsg_shifted_solve(rsg_ham H, const void *b, void *x, int64_t S, int64_t ld, double zr, double zi,
                             int64_t max_iter, double tol, double *resid_out, int64_t *iters_out, void *stream);

/* Checkpoint and resume of a state block, e.g. part-way through a long
 * propagation.  rsg_states_save writes the S live columns of psi ((P, ld)
 * block of the Hamiltonian's dtype, device memory when psi_on_device != 0,
 * else host) to `path` as a NumPy .npy array of shape (P, S) in library
 * point order (complex64 '<c8' or complex128 '<c16', C order), and writes
 * `path`.json with the point and state counts, the dtype, `step`, `time`
 * and the caller's `seed`.  rsg_states_load reads such a file back into
 * psi, zeroing the columns S..ld-1, and returns the metadata through any
 * non-NULL output pointer (then the .json file must exist and match).
 * With a device block, both wait for all work on the device (every stream)
 * before touching it, and load waits again after the copy, so they need no
 * stream.  The files are written under temporary names and renamed into
 * place: a failed save leaves an earlier checkpoint at `path` intact.
 * Errors: RSG_ERR_ARG for NULL,
 * S outside 1..ld, an unreadable or unwritable file, or a file whose dtype,
 * shape or metadata do not match H and S. */
rsg_status rsg_states_save(rsg_ham H, const char *path, const void *psi, int64_t S, int64_t ld,
                           int psi_on_device, int64_t step, double time, uint64_t seed);
rsg_status rsg_states_load(rsg_ham H, const char *path, void *psi, int64_t S, int64_t ld, int psi_on_device,
                           int64_t *step, double *time, uint64_t *seed);

/* FP64 <psi_s|psi_s> for S states into norms2_out (host, S doubles);
 * synchronises. */
rsg_status rsg_state_norms(rsg_ham H, const void *psi, int64_t S, int64_t ld,
                           double *norms2_out, void *stream);

/* Allocation-free variant of rsg_state_norms.  The paper has no counterpart:
 * this is an interface for callers that cannot let the library allocate
 * device memory -- code whose memory belongs to another allocator (a
 * framework's caching allocator or a fixed pool that accounts for every
 * byte) and latency-critical loops where cudaMalloc/cudaFree would
 * synchronise the whole device.  Writes <psi_s|psi_s> (FP64) for S states to
 * norms2_dev (DEVICE array of S doubles, caller-owned, 8-byte aligned);
 * asynchronous on stream.  The partial sums live in one fixed 128 KiB device
 * array inside the library, which every GPU that loads the library holds
 * until the process exits; hence S <= 128 (larger S: RSG_ERR_UNSUPPORTED).
 * No cudaMalloc, cudaFree or allocating library routine is called.  All
 * calls share that array: calls that can overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  The first
 * call on each device looks up the array's device address with that device
 * current; make that first call before any stream capture. */
rsg_status rsg_state_norms_noalloc(rsg_ham H, const void *psi, int64_t S, int64_t ld,
                                   double *norms2_dev, void *stream);

/* Quantum-optimal-control gradient (Sec. "Quantum optimal control",
 * Eq. (qoctgradient) and the costate equations), discrete adjoint of the
 * propagator above for ONE state: J = |<target|psi(T)>|^2 with psi(0) =
 * psi0 (device, P complex values), the control eps[k] (host, nsteps) along
 * dir entering as eps_k dir.r on interval k.  grad_out[k] = dJ/d eps_k
 * (host, nsteps doubles), *J_out = J.  The forward states are checkpointed
 * every checkpoint_every intervals and recomputed per segment; the Taylor
 * powers of one interval are kept so that the gradient costs three forward
 * propagations in Hamiltonian applications.  Synchronises. */
rsg_status rsg_control_gradient(rsg_ham H, const void *psi0, const void *target,
                                int64_t nsteps, double dt, rsg_scheme scheme,
                                int nsub, const double *eps, const double dir[3],
                                int checkpoint_every, double *J_out,
                                double *grad_out, void *stream);

/* Optimal control loop (Sec. "Quantum optimal control": the gradient of
 * Eq. (qoctgradient) drives a gradient-based optimiser; the paper uses
 * conjugate-gradient and BFGS schemes): maximises J = |<target|psi(T)>|^2
 * over the piecewise-constant control eps (host, nsteps doubles: in, the
 * starting field; out, the best field found) by limited-memory BFGS
 * (memory 8) on -J with an Armijo backtracking line search.  Every
 * evaluation is one rsg_control_gradient call with the same psi0, target,
 * nsteps, dt, scheme, nsub, dir and checkpoint_every.  Stops after max_iter
 * accepted steps, when max_k |dJ/deps_k| <= gtol, or when no step along the
 * search direction increases J.  *J_out = J at the returned field; J_hist
 * (host, max_iter + 1 doubles, may be NULL) receives J at the start and
 * after each accepted step (non-decreasing); iters_out / evals_out (may be
 * NULL) the accepted steps and the gradient evaluations.  Synchronises.
 * Errors: as rsg_control_gradient; RSG_ERR_ARG for max_iter < 0 or gtol < 0;
 * RSG_ERR_NONFINITE if J is not finite. */
rsg_status rsg_control_optimize(rsg_ham H, const void *psi0, const void *target, int64_t nsteps, double dt,
                                rsg_scheme scheme, int nsub, double *eps, const double dir[3],
                                int checkpoint_every, int64_t max_iter, double gtol, double *J_out,
                                double *J_hist, int64_t *iters_out, int64_t *evals_out, void *stream);

/* The optimal control loop over a linear parametrisation of the field
 * (Sec. "Quantum optimal control": the parameters that shape the field can
 * be, for example, the Fourier coefficients of its amplitude):
 * eps_k = sum_m basis[k * nparam + m] u_m, and the gradient in u is
 * B^T dJ/deps.  basis: host, nsteps x nparam, row-major, read only (e.g.
 * from rsg_fourier_basis).  u: host, nparam; in, the start; out, the
 * optimum.  Everything else as rsg_control_optimize (J_hist: max_iter + 1
 * values).  Errors: as rsg_control_optimize; RSG_ERR_ARG for nparam < 1 or
 * a non-finite basis value. */
rsg_status rsg_control_optimize_basis(rsg_ham H, const void *psi0, const void *target, int64_t nsteps,
                                      double dt, rsg_scheme scheme, int nsub, int64_t nparam,
                                      const double *basis, double *u, const double dir[3],
                                      int checkpoint_every, int64_t max_iter, double gtol, double *J_out,
                                      double *J_hist, int64_t *iters_out, int64_t *evals_out, void *stream);

/* Fourier (sine-series) basis for rsg_control_optimize_basis: mode m =
 * 1..nparam of a field that vanishes at t = 0 and t = T = nsteps dt,
 * sin(m pi t / T), sampled at the interval midpoints t = (k + 1/2) dt:
 * basis_out[k * nparam + (m - 1)] (host, nsteps x nparam).  The highest
 * frequency is nparam pi / T.  Errors: RSG_ERR_ARG for NULL, nsteps < 1
 * or nparam < 1. */
rsg_status rsg_fourier_basis(int64_t nsteps, int64_t nparam, double *basis_out);

/* -------------------------------------------------------------- batches ---
 * Many independent systems (Sec. "Parallelization, optimizations and graphics processing units": groups of states as the
 * unit of work) propagated together.  hams: nsys Hamiltonians (all
 * complex64, zero ghosts, no mask or complex scaling; otherwise
 * RSG_ERR_UNSUPPORTED), S[i] >= 1 states per system.  The handles must
 * outlive the batch.  RSG_ERR_UNSUPPORTED also when a system has P * ld_i
 * >= 2^31 or more than 32000 points along x. */
rsg_status rsg_batch_create(const rsg_ham *hams, const int64_t *S, int nsys,
                            rsg_batch *out);
/* psis[i]: device (P_i, ld_i) block, 16-byte aligned, with ld_i = S[i]
 * rounded up to even (RSG_ERR_ARG otherwise).  Same step rule as
 * rsg_propagate_steps with no field and nsub = 1.  One time step is a
 * captured CUDA graph, replayed nsteps times on an internal stream ordered
 * after `stream`: by default one persistent launch (k_batch_step) that runs
 * every Horner stage of every system from a queue of work items (projector
 * coefficients per atom, stencil tile segments, projector terms), each item
 * waiting, with a bound, for the items of its own system it depends on.
 * gs_every > 0 re-orthonormalises every system every gs_every steps.  The
 * call returns after the steps complete; RSG_ERR_TIMEOUT if a bounded wait
 * of the step gave up (the states are then undefined, the context stays
 * usable). */
rsg_status rsg_batch_propagate(rsg_batch b, void *const *psis, int64_t nsteps,
                               double dt, rsg_scheme scheme, int gs_every,
                               void *stream);
/* Batch knobs; unknown keys or values give RSG_ERR_ARG.
 *   "persistent": 1 (default) the persistent step kernel; 0 one launch per
 *       Horner stage and kernel (projector coefficients, their reduction,
 *       stencil, projector terms), which propagates the systems one by one
 *       when any has S > 16 or the projector sets differ in size.
 *   "zseg": planes per tile segment of the persistent step (8..128, default
 *       96; RSG_ERR_UNSUPPORTED if the segment does not fit in shared memory).
 *   "wait_limit": polls of one dependency wait before it gives up (each
 *       about 0.5 us; default 2^22).
 *   "tile_variants": bit (ls / 2 - 1) set selects tile variant 1 for the
 *       systems whose staged records hold ls = min(ld, 16) values; only
 *       ls = 14 has one (16 value lanes on a 16 x 6 tile instead of one
 *       lane per value on 18 x 6), other bits are accepted and ignored;
 *       default 0.
 *   "debug_stall": 1 makes system 0 wait for a stencil item that never comes,
 *       so that the step's bounded waits run out (a test of that path).
 * rsg_batch_get_option also reads "batched", "launches_per_step",
 * "items_per_stage" and "blocks" (persistent blocks per launch). */
rsg_status rsg_batch_set_option(rsg_batch b, const char *name, int64_t value);
rsg_status rsg_batch_get_option(rsg_batch b, const char *name, int64_t *value);
/* Batch autotuner: times steps of the given scheme and dt on device copies
 * of psis (psis are read, not changed; the copies are freed before return)
 * for the per-stage launches and the persistent step, and for the persistent
 * step its segment length ("zseg" 48, 64, 96, 128) and the tile variant of
 * the systems with 14 values per point; keeps
 * the fastest and returns its time per step in *best_ms (may be NULL).
 * Synchronises.  Errors as rsg_batch_propagate. */
rsg_status rsg_batch_autotune(rsg_batch b, void *const *psis, double dt, rsg_scheme scheme, void *stream,
                              double *best_ms);
rsg_status rsg_batch_destroy(rsg_batch b);

/* Tuning knobs (kernel tile shapes); unknown keys give RSG_ERR_ARG.
 * Keys: "kernel" (0 = shared-memory staged z-march with cp.async, 1 = one
 * thread per point and vector, 2 = z-march through L1, 3 = z-march with
 * plane tiles gathered by the TMA, 4 = the staged z-march with each tile
 * row segment copied by one TMA box and off-row entries zeroed in shared
 * memory; needs cv = 2, else kernel 0 runs; 5 = the staged z-march with
 * register blocking, complex64 only: one complex value at 2 x 2 points per
 * thread, 16 x 16 tiles with 256 threads or 16 x 12 with 192, else kernel 0
 * runs), "rx" (points per thread along
 * x: 1, 2 or 4; the staged kernel uses 1 or 2), "ty" (rows per
 * tile: 1, 2, 4, 8 or 16), "zseg" (planes per z segment, 1..256; kernels 2
 * and 3 use at most 120), "cv"
 * (staged kernel: 16-byte vectors per point per block, 1, 2, 4 or 8),
 * "threads" (staged kernels: 256 or 512 threads per block; kernel 5: 256
 * gives 16 x 16 tiles, any other value 16 x 12 tiles with 192 threads).
 * Defaults: complex64 runs kernel 5 with 192 threads, 3 stages and 150-plane
 * z segments, complex128 kernel 1; kernels 0, 3 and 4 default to 256
 * threads, cv 2; 160 threads give kernel 5 16 x 10 tiles, three blocks per
 * SM (z segments up to 96 planes keep the three in shared memory).
 * "stages" (staged kernels: shared-memory pipeline depth, 3 or 4 for
 * kernel 0 and for kernel 5 with 192 threads (256 and 160 threads use 3);
 * kernel 4 uses 4, or 5 when set to 5, with 256 threads and 6 with 512),
 * "blocks_per_sm" (staged kernel with 256 threads: register budget for 2 or
 * 3 resident blocks per SM), "adjoint_keep_powers" (rsg_control_gradient: 1 keeps the Taylor powers of
 * a whole checkpoint segment, 0 recomputes them per interval, -1 = choose by
 * free device memory, the default), "adjoint_merge" (rsg_control_gradient
 * with kept powers: 1 runs the costate sweep of a segment and the recompute
 * sweep of the segment before it as two-column launches, 0 one after the
 * other, -1 = 1 when the two banks of two-column blocks fit in half the free
 * memory, the default), "proj_overlap" (1: the projector
 * coefficients of each application run on an internal side stream next to
 * the stencil, which does not read them, and the projector terms after the
 * stencil wait for them; 0, the default: all on the caller's stream).
 * A shape whose shared memory does not fit the SM fails with RSG_ERR_CUDA. */
rsg_status rsg_ham_set_option(rsg_ham H, const char *key, int64_t value);

/* Autotuner: times one Horner stage of H on psi (device, read only) into
 * work (device, same shape, caller-owned scratch) for every candidate stencil
 * configuration (the one-thread-per-value kernel and the two staged kernels
 * in several block shapes and z-segment lengths), keeps the fastest as H's
 * configuration and returns its time per stage in *best_ms (may be NULL).
 * The choice depends on the mesh, S and ld; rerun it when they change.
 * Synchronises. */
rsg_status rsg_ham_autotune(rsg_ham H, const void *psi, void *work, int64_t S, int64_t ld, void *stream,
                            double *best_ms);

/* Reads an option set above, or "last_kernel": the stencil kernel (0..5, or
 * 6 for the complex-scaled operator)
 * that the last Hamiltonian application actually ran (-1 before any), after
 * automatic fallbacks (small problems, TMA unavailable). */
rsg_status rsg_ham_get_option(rsg_ham H, const char *key, int64_t *value);

/* Measurement hooks.  rsg_ham_profile(H, 1) starts recording a CUDA event
 * pair around every stencil-kernel launch of H (on the stream it is
 * launched on); 0 stops.  rsg_ham_kernel_stats waits for the recorded
 * events, returns the summed stencil-kernel time in ms, the number of those
 * launches, their algorithmic bytes (the unique state, potential, grid-table
 * and projector bytes each launch must move; see the design notes) and the
 * number of kernel launches of any kind H issued since the last call, then
 * resets all four.  Any output pointer may be NULL. */
rsg_status rsg_ham_profile(rsg_ham H, int enable);
rsg_status rsg_ham_kernel_stats(rsg_ham H, double *kernel_ms, int64_t *kernel_launches,
                                double *kernel_bytes, int64_t *all_launches);

/* Failure-path support (no counterpart in the paper).
 * rsg_selftest_bounded_wait runs the bounded-wait path of the pipelined
 * stencil kernels on purpose: one warp waits on an mbarrier phase that
 * cannot complete, polling `polls` times (1..65536, each poll suspending
 * for at most about a microsecond), records the timeout in the handle's
 * status word and returns; the call then reports RSG_ERR_TIMEOUT, and the
 * handle and the CUDA context stay usable.  Synchronises the stream.
 * rsg_debug_fail_allocations(n) makes the library's next n device
 * allocations fail as if the device were out of memory (RSG_ERR_OOM from
 * the call that needed them); 0 clears it.  Errors: RSG_ERR_ARG for polls
 * outside 1..65536 or n < 0. */
rsg_status rsg_selftest_bounded_wait(rsg_ham H, int polls, void *stream);
rsg_status rsg_debug_fail_allocations(int n);

/* Diagnostics on stderr: 0 silent (default), 1 every error status with
 * its message, 2 also the stencil-kernel fallbacks (small problems, block
 * shapes a kernel does not take).  The environment variable RSG_LOG_LEVEL
 * sets the initial level.  Errors: RSG_ERR_ARG for a level outside 0..2. */
rsg_status rsg_set_log_level(int level);

/* Thread-local description of the last error (empty if none). */
const char *rsg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RSG_H */
