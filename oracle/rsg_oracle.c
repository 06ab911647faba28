/*
 * rsg_oracle.c -- plain, slow, FP64 CPU oracle for the real-space-grid
 * Hamiltonian, its Taylor-4 real-time propagator and the discrete adjoint
 * gradient of a dipole-control objective.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every loop follows the textbook statement of the step it implements, in
 * the order written, with OpenMP `parallel for` over independent points as
 * the only concession to speed.  Sources (arXiv:1501.05654):
 *   - Sec. 1 (introduction): fields sampled on a uniform real-space grid,
 *     integrals become grid sums, derivatives become high-order finite
 *     differences; the error is controlled by the spacing and the box.
 *   - Sec. "Magnetic response and gauge invariance in real-space grids"/hyper-virial passage: pseudopotentials enter
 *     as a non-local operator v_nl (separable projectors here).
 *   - Sec. "Quantum optimal control", Eq. (qoctgradient) and the costate
 *     equations: gradient = 2 Im int <chi| dH/du |psi> dt, costate
 *     propagated backwards with the forward propagators.
 *   - Sec. "Parallelization, optimizations and graphics processing units": a block of states is the basic object; fields are
 *     linear arrays plus tables describing the grid.
 *
 * Readings the paper leaves open (restated in the design notes):
 *   - Laplacian: 8th-order central second difference, radius 4 per axis
 *     (25-point star), c = (-205/72, 8/5, -1/5, 8/315, -1/560) / h^2.
 *   - Kinetic operator -1/2 nabla^2 (atomic units).
 *   - Boundary: ghost values outside the mesh are zero (ZERO).  A test-only
 *     ODD mode (cube/box) uses antisymmetric images about walls one spacing
 *     outside the mesh, which makes sines exact eigenvectors.
 *   - Inner product <f|g> = h^3 sum_p conj(f_p) g_p.
 *   - Projectors p_ai(r) = Y_i(r - R_a) exp(-|r-R_a|^2/(2 beta^2)) on mesh
 *     points with |r - R_a| <= r_c, Y in {1; x,y,z; xy,yz,zx,x^2-y^2,
 *     3z^2-r^2}, each scaled so that h^3 sum p^2 = 1.
 *   - Taylor-4: T(tau) = sum_{n=0..4} (-i tau H)^n / n!.
 *   - The control field is piecewise constant, eps_k on [t_k, t_k + dt).
 *     Exponential midpoint uses H(t_k + dt/2); ETRS uses H(t_k) for the
 *     first half step and H(t_{k+1}) (left limit, same eps_k) for the second.
 *
 * Point order: x-major (i slowest, k fastest) over the mesh -- deliberately
 * not the CUDA library's order; tests match points by lattice coordinates.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORC_CUBE = 0, ORC_SPHERE = 1, ORC_BOX = 2 };
enum { ORC_ZERO = 0, ORC_ODD = 1 };
enum { ORC_EXPMID = 0, ORC_ETRS = 1 };

/* 8th-order second-derivative weights, |k| = 0..4 (times 1/h^2). */
static const double FD_C[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0,
                                8.0 / 315.0, -1.0 / 560.0};

typedef struct {
    int shape, bc;
    double h;
    int32_t lo[3], hi[3];   /* inclusive lattice bounds of the bounding box */
    int32_t ext[3];         /* hi - lo + 1 */
    double origin[3];       /* position of lattice coordinate (0,0,0) */
    int64_t P;
    int32_t *ijk;           /* P x 3 lattice coordinates */
    int64_t *lookup;        /* dense bbox -> point index, -1 outside */
} orc_mesh;

typedef struct {
    int64_t npts;
    int nproj;
    int64_t *pt;            /* mesh point indices inside the sphere */
    double *p;              /* nproj x npts projector values */
    double *hm;             /* nproj x nproj coupling matrix */
} orc_atom;

typedef struct {
    orc_mesh *m;
    double *V;              /* local potential, P */
    int natoms;
    orc_atom *atoms;
} orc_ham;

/* ------------------------------------------------------------------------ */
/* mesh                                                                      */
/* ------------------------------------------------------------------------ */

static int64_t lk_index(const orc_mesh *m, int32_t i, int32_t j, int32_t k)
{
    if (i < m->lo[0] || i > m->hi[0] || j < m->lo[1] || j > m->hi[1] ||
        k < m->lo[2] || k > m->hi[2])
        return -1;
    int64_t a = i - m->lo[0], b = j - m->lo[1], c = k - m->lo[2];
    return m->lookup[(a * m->ext[1] + b) * m->ext[2] + c];
}

static int in_shape(int shape, int32_t i, int32_t j, int32_t k, int64_t r2max)
{
    if (shape == ORC_SPHERE)
        return (int64_t)i * i + (int64_t)j * j + (int64_t)k * k <= r2max;
    return 1;
}

/* Cube/box: lattice i = 0..n-1 at x = (i - (n-1)/2) h.
 * Sphere: lattice i in [-M, M] at x = i h, kept iff i^2+j^2+k^2 <= (R/h)^2
 * (integer test, boundary inclusive). */
void *orc_mesh_new(int shape, const int32_t *n, double radius, double h, int bc)
{
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    m->shape = shape;
    m->bc = bc;
    m->h = h;
    int64_t r2max = 0;
    if (shape == ORC_SPHERE) {
        double q = radius / h;
        r2max = (int64_t)floor(q * q + 1e-6);
        int32_t M = (int32_t)floor(sqrt((double)r2max) + 1e-9);
        for (int d = 0; d < 3; d++) {
            m->lo[d] = -M;
            m->hi[d] = M;
            m->origin[d] = 0.0;
        }
    } else {
        for (int d = 0; d < 3; d++) {
            int32_t nd = (shape == ORC_CUBE) ? n[0] : n[d];
            m->lo[d] = 0;
            m->hi[d] = nd - 1;
            m->origin[d] = -0.5 * (double)(nd - 1) * h;
        }
    }
    for (int d = 0; d < 3; d++) m->ext[d] = m->hi[d] - m->lo[d] + 1;
    /* image walls: one reflection reaches every neighbour's image only with
     * at least 4 points along each axis */
    if (bc == ORC_ODD && (m->ext[0] < 4 || m->ext[1] < 4 || m->ext[2] < 4)) {
        free(m);
        return NULL;
    }
    int64_t nbox = (int64_t)m->ext[0] * m->ext[1] * m->ext[2];
    m->lookup = (int64_t *)malloc(sizeof(int64_t) * nbox);
    int64_t P = 0;
    for (int32_t i = m->lo[0]; i <= m->hi[0]; i++)
        for (int32_t j = m->lo[1]; j <= m->hi[1]; j++)
            for (int32_t k = m->lo[2]; k <= m->hi[2]; k++) {
                int64_t a = i - m->lo[0], b = j - m->lo[1], c = k - m->lo[2];
                int64_t at = (a * m->ext[1] + b) * m->ext[2] + c;
                if (in_shape(shape, i, j, k, r2max))
                    m->lookup[at] = P++;
                else
                    m->lookup[at] = -1;
            }
    m->P = P;
    m->ijk = (int32_t *)malloc(sizeof(int32_t) * 3 * (P ? P : 1));
    for (int32_t i = m->lo[0]; i <= m->hi[0]; i++)
        for (int32_t j = m->lo[1]; j <= m->hi[1]; j++)
            for (int32_t k = m->lo[2]; k <= m->hi[2]; k++) {
                int64_t p = lk_index(m, i, j, k);
                if (p >= 0) {
                    m->ijk[3 * p] = i;
                    m->ijk[3 * p + 1] = j;
                    m->ijk[3 * p + 2] = k;
                }
            }
    return m;
}

int64_t orc_mesh_npoints(void *mv) { return ((orc_mesh *)mv)->P; }

void orc_mesh_ijk(void *mv, int32_t *out)
{
    orc_mesh *m = (orc_mesh *)mv;
    memcpy(out, m->ijk, sizeof(int32_t) * 3 * m->P);
}

void orc_mesh_xyz(void *mv, double *out)
{
    orc_mesh *m = (orc_mesh *)mv;
    for (int64_t p = 0; p < m->P; p++)
        for (int d = 0; d < 3; d++)
            out[3 * p + d] = m->origin[d] + m->h * (double)m->ijk[3 * p + d];
}

void orc_mesh_free(void *mv)
{
    orc_mesh *m = (orc_mesh *)mv;
    if (!m) return;
    free(m->ijk);
    free(m->lookup);
    free(m);
}

/* Value of state s at lattice site (i,j,k), applying the boundary rule. */
static cplx site_value(const orc_mesh *m, const cplx *psi, int64_t S,
                       int64_t s, int32_t c[3])
{
    int64_t q = lk_index(m, c[0], c[1], c[2]);
    if (q >= 0) return psi[q * S + s];
    if (m->bc != ORC_ODD || m->shape == ORC_SPHERE) return 0.0;
    /* ODD: reflect every out-of-range axis about the wall one spacing
     * outside the mesh (at lo-1 and hi+1) and flip the sign per reflection. */
    int32_t r[3] = {c[0], c[1], c[2]};
    double sign = 1.0;
    for (int d = 0; d < 3; d++) {
        if (r[d] < m->lo[d]) {
            r[d] = 2 * (m->lo[d] - 1) - r[d];
            sign = -sign;
        } else if (r[d] > m->hi[d]) {
            r[d] = 2 * (m->hi[d] + 1) - r[d];
            sign = -sign;
        }
        if (r[d] < m->lo[d] || r[d] > m->hi[d]) return 0.0; /* on a wall */
    }
    q = lk_index(m, r[0], r[1], r[2]);
    return q >= 0 ? sign * psi[q * S + s] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Hamiltonian                                                               */
/* ------------------------------------------------------------------------ */

void *orc_ham_new(void *mv, const double *V)
{
    orc_ham *H = (orc_ham *)calloc(1, sizeof(orc_ham));
    H->m = (orc_mesh *)mv;
    H->V = (double *)malloc(sizeof(double) * (H->m->P ? H->m->P : 1));
    memcpy(H->V, V, sizeof(double) * H->m->P);
    return H;
}

static void free_atoms(orc_ham *H)
{
    for (int a = 0; a < H->natoms; a++) {
        free(H->atoms[a].pt);
        free(H->atoms[a].p);
        free(H->atoms[a].hm);
    }
    free(H->atoms);
    H->atoms = NULL;
    H->natoms = 0;
}

void orc_ham_free(void *hv)
{
    orc_ham *H = (orc_ham *)hv;
    if (!H) return;
    free_atoms(H);
    free(H->V);
    free(H);
}

/* Real solid-harmonic polynomial i (0..8) at displacement (x,y,z). */
static double solid_harmonic(int i, double x, double y, double z)
{
    switch (i) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * y;
    case 5: return y * z;
    case 6: return z * x;
    case 7: return x * x - y * y;
    case 8: return 3.0 * z * z - (x * x + y * y + z * z);
    }
    return 0.0;
}

/* Builds, for every atom, its sphere {p : |r_p - R_a| <= r_c}, the sampled
 * projectors (Gaussian radial part times real solid harmonics, discretely
 * normalised to h^3 sum p^2 = 1) and copies the coupling matrix h_a. */
void orc_ham_set_projectors(void *hv, int natoms, const double *centres,
                            const double *rcut, const int32_t *lmax,
                            const double *beta, const double *hmats)
{
    orc_ham *H = (orc_ham *)hv;
    orc_mesh *m = H->m;
    free_atoms(H);
    H->natoms = natoms;
    H->atoms = (orc_atom *)calloc(natoms ? natoms : 1, sizeof(orc_atom));
    double h3 = m->h * m->h * m->h;
    int64_t hoff = 0;
    for (int a = 0; a < natoms; a++) {
        orc_atom *A = &H->atoms[a];
        A->nproj = (lmax[a] + 1) * (lmax[a] + 1);
        int64_t n = 0;
        for (int64_t p = 0; p < m->P; p++) {
            double d2 = 0.0;
            for (int d = 0; d < 3; d++) {
                double x = m->origin[d] + m->h * m->ijk[3 * p + d] - centres[3 * a + d];
                d2 += x * x;
            }
            if (d2 <= rcut[a] * rcut[a]) n++;
        }
        A->npts = n;
        A->pt = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
        A->p = (double *)malloc(sizeof(double) * A->nproj * (n ? n : 1));
        n = 0;
        for (int64_t p = 0; p < m->P; p++) {
            double r[3], d2 = 0.0;
            for (int d = 0; d < 3; d++) {
                r[d] = m->origin[d] + m->h * m->ijk[3 * p + d] - centres[3 * a + d];
                d2 += r[d] * r[d];
            }
            if (d2 <= rcut[a] * rcut[a]) {
                A->pt[n] = p;
                double g = exp(-d2 / (2.0 * beta[a] * beta[a]));
                for (int i = 0; i < A->nproj; i++)
                    A->p[i * A->npts + n] = solid_harmonic(i, r[0], r[1], r[2]) * g;
                n++;
            }
        }
        for (int i = 0; i < A->nproj; i++) {
            double ss = 0.0;
            for (int64_t q = 0; q < A->npts; q++)
                ss += A->p[i * A->npts + q] * A->p[i * A->npts + q];
            double nrm = sqrt(h3 * ss);
            if (nrm > 0.0)
                for (int64_t q = 0; q < A->npts; q++) A->p[i * A->npts + q] /= nrm;
        }
        A->hm = (double *)malloc(sizeof(double) * A->nproj * A->nproj);
        memcpy(A->hm, hmats + hoff, sizeof(double) * A->nproj * A->nproj);
        hoff += A->nproj * A->nproj;
    }
}

/* The same non-local term from projector values the caller has sampled:
 * atom a covers npts[a] mesh points point_idx[...] (concatenated over
 * atoms) with nproj[a] values per point (pvals, point-major), taken as
 * given, and the nproj x nproj coupling matrix h_a (concatenated). */
void orc_ham_set_projectors_raw(void *hv, int natoms, const int64_t *npts, const int64_t *point_idx,
                                const int32_t *nproj, const double *pvals, const double *hmats)
{
    orc_ham *H = (orc_ham *)hv;
    free_atoms(H);
    H->natoms = natoms;
    H->atoms = (orc_atom *)calloc(natoms ? natoms : 1, sizeof(orc_atom));
    int64_t off = 0, voff = 0, hoff = 0;
    for (int a = 0; a < natoms; a++) {
        orc_atom *A = &H->atoms[a];
        int64_t n = npts[a];
        A->npts = n;
        A->nproj = nproj[a];
        A->pt = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
        A->p = (double *)malloc(sizeof(double) * A->nproj * (n ? n : 1));
        for (int64_t k = 0; k < n; k++) {
            A->pt[k] = point_idx[off + k];
            for (int i = 0; i < A->nproj; i++) A->p[i * n + k] = pvals[voff + k * A->nproj + i];
        }
        A->hm = (double *)malloc(sizeof(double) * A->nproj * A->nproj);
        memcpy(A->hm, hmats + hoff, sizeof(double) * A->nproj * A->nproj);
        off += n;
        voff += n * A->nproj;
        hoff += (int64_t)A->nproj * A->nproj;
    }
}

int64_t orc_ham_atom_npoints(void *hv, int a) { return ((orc_ham *)hv)->atoms[a].npts; }
int orc_ham_atom_nproj(void *hv, int a) { return ((orc_ham *)hv)->atoms[a].nproj; }

void orc_ham_atom_values(void *hv, int a, int64_t *pts, double *vals)
{
    orc_atom *A = &((orc_ham *)hv)->atoms[a];
    memcpy(pts, A->pt, sizeof(int64_t) * A->npts);
    memcpy(vals, A->p, sizeof(double) * A->npts * A->nproj);
}

/* Position component along dir, used by the dipole term eps * (dir . r). */
static double dipole_coord(const orc_mesh *m, int64_t p, const double *dir)
{
    double s = 0.0;
    for (int d = 0; d < 3; d++)
        s += dir[d] * (m->origin[d] + m->h * m->ijk[3 * p + d]);
    return s;
}

/* (H psi)[p,s] for one point and state: kinetic, local and dipole parts. */
static cplx local_part(const orc_ham *H, double eps, const double *dir,
                       const cplx *psi, int64_t S, int64_t p, int64_t s)
{
    const orc_mesh *m = H->m;
    double ih2 = 1.0 / (m->h * m->h);
    cplx lap = 0.0;
    for (int d = 0; d < 3; d++) {
        for (int k = -4; k <= 4; k++) {
            int32_t c[3] = {m->ijk[3 * p], m->ijk[3 * p + 1], m->ijk[3 * p + 2]};
            c[d] += k;
            lap += FD_C[abs(k)] * ih2 * site_value(m, psi, S, s, c);
        }
    }
    double v = H->V[p];
    if (dir) v += eps * dipole_coord(m, p, dir);
    return -0.5 * lap + v * psi[p * S + s];
}

/* Non-local coefficients d[a][i][s] = sum_j h_a[i][j] <p_aj|psi_s>. */
static cplx *nonlocal_coeffs(const orc_ham *H, const cplx *psi, int64_t S)
{
    int64_t tot = 0;
    for (int a = 0; a < H->natoms; a++) tot += (int64_t)H->atoms[a].nproj * S;
    cplx *d = (cplx *)calloc(tot ? tot : 1, sizeof(cplx));
    double h3 = H->m->h * H->m->h * H->m->h;
    int64_t off = 0;
    for (int a = 0; a < H->natoms; a++) {
        const orc_atom *A = &H->atoms[a];
        cplx *c = (cplx *)calloc(A->nproj * S, sizeof(cplx));
        for (int j = 0; j < A->nproj; j++)
            for (int64_t s = 0; s < S; s++) {
                cplx acc = 0.0;
                for (int64_t q = 0; q < A->npts; q++)
                    acc += A->p[j * A->npts + q] * psi[A->pt[q] * S + s];
                c[j * S + s] = h3 * acc;
            }
        for (int i = 0; i < A->nproj; i++)
            for (int64_t s = 0; s < S; s++) {
                cplx acc = 0.0;
                for (int j = 0; j < A->nproj; j++)
                    acc += A->hm[i * A->nproj + j] * c[j * S + s];
                d[off + i * S + s] = acc;
            }
        free(c);
        off += (int64_t)A->nproj * S;
    }
    return d;
}

/* hpsi = H(eps) psi for all P x S values (states fastest). */
void orc_apply(void *hv, double eps, const double *dir, const cplx *psi,
               cplx *hpsi, int64_t S)
{
    const orc_ham *H = (const orc_ham *)hv;
    int64_t P = H->m->P;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; p++)
        for (int64_t s = 0; s < S; s++)
            hpsi[p * S + s] = local_part(H, eps, dir, psi, S, p, s);
    if (H->natoms == 0) return;
    cplx *d = nonlocal_coeffs(H, psi, S);
    int64_t off = 0;
    for (int a = 0; a < H->natoms; a++) {
        const orc_atom *A = &H->atoms[a];
        for (int64_t q = 0; q < A->npts; q++)
            for (int64_t s = 0; s < S; s++) {
                cplx acc = 0.0;
                for (int i = 0; i < A->nproj; i++)
                    acc += A->p[i * A->npts + q] * d[off + i * S + s];
                hpsi[A->pt[q] * S + s] += acc;
            }
        off += (int64_t)A->nproj * S;
    }
    free(d);
}

/* Complex-scaled operator (Sec. "Complex scaling and resonances": r -> r
 * e^{i theta} turns the kinetic term into -1/2 e^{-2 i theta} lap and the
 * potential into V(r e^{i theta})): hpsi = -1/2 e^{-2 i theta} lap psi +
 * vtheta psi, with vtheta the caller's values of V(r e^{i theta}) on the
 * mesh (no projectors, no field).  The Laplacian is the mesh's 8th-order
 * stencil with the mesh's boundary rule. */
static cplx scaled_point(const orc_mesh *m, cplx rot, const cplx *vtheta, const cplx *psi, int64_t S,
                         int64_t p, int64_t s)
{
    const double ih2 = 1.0 / (m->h * m->h);
    cplx lap = 0.0;
    for (int d = 0; d < 3; d++)
        for (int k = -4; k <= 4; k++) {
            int32_t c[3] = {m->ijk[3 * p], m->ijk[3 * p + 1], m->ijk[3 * p + 2]};
            c[d] += k;
            lap += FD_C[abs(k)] * ih2 * site_value(m, psi, S, s, c);
        }
    return -0.5 * rot * lap + vtheta[p] * psi[p * S + s];
}

void orc_apply_scaled(void *mv, double theta, const cplx *vtheta, const cplx *psi, cplx *hpsi,
                      int64_t S)
{
    const orc_mesh *m = (const orc_mesh *)mv;
    const cplx rot = cexp(-2.0 * I * theta);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < m->P; p++)
        for (int64_t s = 0; s < S; s++) hpsi[p * S + s] = scaled_point(m, rot, vtheta, psi, S, p, s);
}

/* (H_theta psi) at nsamp chosen (point, state) pairs only; for full-size checks. */
void orc_apply_scaled_sampled(void *mv, double theta, const cplx *vtheta, const cplx *psi, int64_t S,
                              int64_t nsamp, const int64_t *pidx, const int64_t *sidx, cplx *out)
{
    const orc_mesh *m = (const orc_mesh *)mv;
    const cplx rot = cexp(-2.0 * I * theta);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nsamp; t++) out[t] = scaled_point(m, rot, vtheta, psi, S, pidx[t], sidx[t]);
}

/* Taylor-4 exponential of the complex-scaled operator, by explicit terms
 * (as orc_taylor4): out = sum_{n=0..4} (-i tau H_theta)^n psi / n!. */
void orc_taylor4_scaled(void *mv, double theta, const cplx *vtheta, double tau, const cplx *psi, cplx *out,
                        int64_t S)
{
    const orc_mesh *m = (const orc_mesh *)mv;
    int64_t N = m->P * S;
    cplx *term = (cplx *)malloc(sizeof(cplx) * (N ? N : 1));
    cplx *next = (cplx *)malloc(sizeof(cplx) * (N ? N : 1));
    memcpy(term, psi, sizeof(cplx) * N);
    memcpy(out, psi, sizeof(cplx) * N);
    for (int n = 1; n <= 4; n++) {
        orc_apply_scaled(mv, theta, vtheta, term, next, S);
        cplx f = -I * tau / (double)n;
        for (int64_t t = 0; t < N; t++) {
            term[t] = f * next[t];
            out[t] += term[t];
        }
    }
    free(term);
    free(next);
}

/* nsteps time steps of dt with the (time-independent) complex-scaled
 * operator: exponential midpoint T(dt), or ETRS T(dt/2) T(dt/2). */
void orc_propagate_scaled(void *mv, double theta, const cplx *vtheta, cplx *psi, int64_t S, int64_t nsteps,
                          double dt, int scheme)
{
    const orc_mesh *m = (const orc_mesh *)mv;
    int64_t N = m->P * S;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (N ? N : 1));
    for (int64_t k = 0; k < nsteps; k++) {
        if (scheme == 0) {
            orc_taylor4_scaled(mv, theta, vtheta, dt, psi, tmp, S);
            memcpy(psi, tmp, sizeof(cplx) * N);
        } else {
            orc_taylor4_scaled(mv, theta, vtheta, 0.5 * dt, psi, tmp, S);
            orc_taylor4_scaled(mv, theta, vtheta, 0.5 * dt, tmp, psi, S);
        }
    }
    free(tmp);
}

/* (H psi) at nsamp chosen (point, state) pairs only; for full-size checks. */
void orc_apply_sampled(void *hv, double eps, const double *dir, const cplx *psi,
                       int64_t S, int64_t nsamp, const int64_t *pidx,
                       const int64_t *sidx, cplx *out)
{
    const orc_ham *H = (const orc_ham *)hv;
    cplx *d = H->natoms ? nonlocal_coeffs(H, psi, S) : NULL;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nsamp; t++) {
        int64_t p = pidx[t], s = sidx[t];
        cplx v = local_part(H, eps, dir, psi, S, p, s);
        int64_t off = 0;
        for (int a = 0; a < H->natoms; a++) {
            const orc_atom *A = &H->atoms[a];
            /* the sphere's point list is ascending: binary search for p */
            int64_t lo = 0, hi = A->npts;
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (A->pt[mid] < p) lo = mid + 1; else hi = mid;
            }
            if (lo < A->npts && A->pt[lo] == p)
                for (int i = 0; i < A->nproj; i++)
                    v += A->p[i * A->npts + lo] * d[off + i * S + s];
            off += (int64_t)A->nproj * S;
        }
        out[t] = v;
    }
    free(d);
}

/* ------------------------------------------------------------------------ */
/* Taylor-4 exponential, explicit term accumulation                         */
/* ------------------------------------------------------------------------ */

/* out = sum_{n=0..4} (-i tau H)^n / n! psi, built term by term:
 * term_0 = psi, term_n = (-i tau / n) H term_{n-1}. */
void orc_taylor4(void *hv, double eps, const double *dir, double tau,
                 const cplx *psi, cplx *out, int64_t S)
{
    const orc_ham *H = (const orc_ham *)hv;
    int64_t N = H->m->P * S;
    cplx *term = (cplx *)malloc(sizeof(cplx) * (N ? N : 1));
    cplx *next = (cplx *)malloc(sizeof(cplx) * (N ? N : 1));
    memcpy(term, psi, sizeof(cplx) * N);
    memcpy(out, psi, sizeof(cplx) * N);
    for (int n = 1; n <= 4; n++) {
        orc_apply(hv, eps, dir, term, next, S);
        cplx f = -I * tau / (double)n;
        for (int64_t t = 0; t < N; t++) {
            term[t] = f * next[t];
            out[t] += term[t];
        }
    }
    free(term);
    free(next);
}

/* ------------------------------------------------------------------------ */
/* norms and Gram-Schmidt                                                    */
/* ------------------------------------------------------------------------ */

static cplx inner(const orc_mesh *m, const cplx *f, const cplx *g, int64_t S,
                  int64_t sf, int64_t sg)
{
    cplx acc = 0.0;
    for (int64_t p = 0; p < m->P; p++) acc += conj(f[p * S + sf]) * g[p * S + sg];
    return m->h * m->h * m->h * acc;
}

void orc_norms2(void *mv, const cplx *psi, int64_t S, double *out)
{
    const orc_mesh *m = (const orc_mesh *)mv;
    for (int64_t s = 0; s < S; s++) out[s] = creal(inner(m, psi, psi, S, s, s));
}

/* Modified Gram-Schmidt in index order with the h^3-weighted product. */
void orc_mgs(void *mv, cplx *psi, int64_t S)
{
    const orc_mesh *m = (const orc_mesh *)mv;
    for (int64_t s = 0; s < S; s++) {
        for (int64_t t = 0; t < s; t++) {
            cplx r = inner(m, psi, psi, S, t, s);
            for (int64_t p = 0; p < m->P; p++) psi[p * S + s] -= r * psi[p * S + t];
        }
        double nrm = sqrt(creal(inner(m, psi, psi, S, s, s)));
        for (int64_t p = 0; p < m->P; p++) psi[p * S + s] /= nrm;
    }
}

/* ------------------------------------------------------------------------ */
/* time stepping                                                             */
/* ------------------------------------------------------------------------ */

/* One control interval k (field eps_k, piecewise constant). */
static void one_step(void *hv, cplx *psi, cplx *tmp, int64_t S, double dt,
                     int scheme, int nsub, double eps, const double *dir)
{
    const orc_ham *H = (const orc_ham *)hv;
    int64_t N = H->m->P * S;
    double tsub = dt / (double)nsub;
    for (int u = 0; u < nsub; u++) {
        if (scheme == ORC_EXPMID) {
            /* psi <- T_{H(t + tsub/2)}(tsub) psi */
            orc_taylor4(hv, eps, dir, tsub, psi, tmp, S);
            memcpy(psi, tmp, sizeof(cplx) * N);
        } else {
            /* psi <- T_{H(t + tsub)}(tsub/2) T_{H(t)}(tsub/2) psi; both
             * Hamiltonians carry the interval's constant field eps_k. */
            orc_taylor4(hv, eps, dir, 0.5 * tsub, psi, tmp, S);
            orc_taylor4(hv, eps, dir, 0.5 * tsub, tmp, psi, S);
        }
    }
}

/* Propagates nsteps intervals.  Every gs_every steps (0 = never) the norm
 * drift max_s |<psi_s|psi_s> - 1| is recorded and the block re-orthonormalised
 * by MGS; the final block is also checked.  drift_out (S) may be NULL. */
void orc_propagate(void *hv, cplx *psi, int64_t S, int64_t nsteps, double dt,
                   int scheme, int nsub, const double *eps, const double *dir,
                   int gs_every, double *drift_out)
{
    const orc_ham *H = (const orc_ham *)hv;
    int64_t N = H->m->P * S;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (N ? N : 1));
    double *n2 = (double *)malloc(sizeof(double) * (S ? S : 1));
    if (drift_out)
        for (int64_t s = 0; s < S; s++) drift_out[s] = 0.0;
    for (int64_t k = 0; k < nsteps; k++) {
        one_step(hv, psi, tmp, S, dt, scheme, nsub, eps ? eps[k] : 0.0, dir);
        int gs_now = gs_every > 0 && (k + 1) % gs_every == 0;
        if (gs_now || k == nsteps - 1) {
            orc_norms2(H->m, psi, S, n2);
            if (drift_out)
                for (int64_t s = 0; s < S; s++)
                    if (fabs(n2[s] - 1.0) > drift_out[s]) drift_out[s] = fabs(n2[s] - 1.0);
        }
        if (gs_now) orc_mgs(H->m, psi, S);
    }
    free(tmp);
    free(n2);
}

/* ------------------------------------------------------------------------ */
/* control objective and discrete adjoint gradient                          */
/* ------------------------------------------------------------------------ */

/* J = |<phi|psi(T)>|^2 for one state (S = 1), forward only. */
double orc_objective(void *hv, const cplx *psi0, const cplx *target,
                     int64_t nsteps, double dt, int scheme, int nsub,
                     const double *eps, const double *dir)
{
    const orc_ham *H = (const orc_ham *)hv;
    int64_t P = H->m->P;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * P);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * P);
    memcpy(psi, psi0, sizeof(cplx) * P);
    for (int64_t k = 0; k < nsteps; k++)
        one_step(hv, psi, tmp, 1, dt, scheme, nsub, eps[k], dir);
    cplx ov = inner(H->m, target, psi, 1, 0, 0);
    free(psi);
    free(tmp);
    return creal(ov * conj(ov));
}

/* Every exponential of interval k is T(tau) with A = -i tau H_k,
 * H_k = H0 + eps_k X, X = dir . r; m of them per interval. */
static void interval_layout(int scheme, int nsub, double dt, int *m, double *tau)
{
    if (scheme == ORC_EXPMID) {
        *m = nsub;
        *tau = dt / nsub;
    } else {
        *m = 2 * nsub;
        *tau = 0.5 * dt / nsub;
    }
}

/* Returns J and fills grad[k] = dJ/d eps_k.
 *
 * Discrete adjoint of psi_{k+1} = U_k psi_k with U_k = T^m:
 *   chi_N = phi <phi|psi_N>,  chi_k = U_k^dagger chi_{k+1},
 *   dJ/d eps_k = 2 Re <chi_{k+1}| dU_k/d eps_k |psi_k>,
 *   dU_k = sum_l T^{m-1-l} dT T^l,
 *   dT   = sum_{n=1..4} 1/n! sum_{j=0..n-1} A^j (-i tau X) A^{n-1-j}.
 * This is the time-discrete form of the gradient 2 Im int <chi|dH/du|psi> dt
 * with the costate carried backwards by the adjoint of the same propagator.
 * T^dagger uses A^dagger = +i tau H (H is real symmetric).
 * States are checkpointed every `checkpoint_every` intervals and recomputed
 * forward within each segment. */
double orc_control_gradient(void *hv, const cplx *psi0, const cplx *target,
                            int64_t nsteps, double dt, int scheme, int nsub,
                            const double *eps, const double *dir,
                            int checkpoint_every, double *grad)
{
    const orc_ham *H = (const orc_ham *)hv;
    const orc_mesh *msh = H->m;
    int64_t P = msh->P;
    size_t vb = sizeof(cplx) * (size_t)P;
    int m;
    double tau;
    interval_layout(scheme, nsub, dt, &m, &tau);
    int K = checkpoint_every > 0 ? checkpoint_every : (int)nsteps;
    int64_t nck = (nsteps + K - 1) / K;

    /* forward pass, saving psi at the start of each segment */
    cplx *ck = (cplx *)malloc(vb * (nck ? nck : 1));
    cplx *psi = (cplx *)malloc(vb);
    cplx *tmp = (cplx *)malloc(vb);
    memcpy(psi, psi0, vb);
    for (int64_t k = 0; k < nsteps; k++) {
        if (k % K == 0) memcpy(ck + (k / K) * P, psi, vb);
        one_step(hv, psi, tmp, 1, dt, scheme, nsub, eps[k], dir);
    }
    cplx ov = inner(msh, target, psi, 1, 0, 0);
    double J = creal(ov * conj(ov));

    /* chi_N = phi <phi|psi_N> */
    cplx *chi = (cplx *)malloc(vb);
    for (int64_t p = 0; p < P; p++) chi[p] = target[p] * ov;

    cplx *seg = (cplx *)malloc(vb * (size_t)(K + 1));   /* psi_k in a segment */
    cplx *psis = (cplx *)malloc(vb * (size_t)(m + 1));  /* T^l psi_k, l=0..m */
    cplx *chis = (cplx *)malloc(vb * (size_t)(m + 1));  /* chi'_l, l=0..m */
    cplx *apow = (cplx *)malloc(vb * 4);                /* A^j psi', j=0..3 */
    cplx *bpow = (cplx *)malloc(vb * 4);                /* (A^dag)^j chi', j=0..3 */
    cplx *hv_t = (cplx *)malloc(vb);
    double *X = (double *)malloc(sizeof(double) * P);
    for (int64_t p = 0; p < P; p++) X[p] = dipole_coord(msh, p, dir);
    double h3 = msh->h * msh->h * msh->h;
    static const double invfact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};

    for (int64_t c = nck - 1; c >= 0; c--) {
        int64_t k0 = c * K, k1 = (k0 + K < nsteps) ? k0 + K : nsteps;
        memcpy(seg, ck + c * P, vb);
        for (int64_t k = k0; k < k1; k++) {
            memcpy(seg + (k - k0 + 1) * P, seg + (k - k0) * P, vb);
            one_step(hv, seg + (k - k0 + 1) * P, tmp, 1, dt, scheme, nsub, eps[k], dir);
        }
        for (int64_t k = k1 - 1; k >= k0; k--) {
            double e = eps[k];
            /* forward exponentials of the interval */
            memcpy(psis, seg + (k - k0) * P, vb);
            for (int l = 0; l < m; l++)
                orc_taylor4(hv, e, dir, tau, psis + l * P, psis + (l + 1) * P, 1);
            /* backward: chi'_m = chi_{k+1}, chi'_l = T^dagger chi'_{l+1} */
            memcpy(chis + m * P, chi, vb);
            for (int l = m - 1; l >= 0; l--)
                orc_taylor4(hv, e, dir, -tau, chis + (l + 1) * P, chis + l * P, 1);
            double g = 0.0;
            for (int l = 0; l < m; l++) {
                /* powers A^j psi'_l and (A^dag)^j chi'_{l+1}, j = 0..3 */
                memcpy(apow, psis + l * P, vb);
                memcpy(bpow, chis + (l + 1) * P, vb);
                for (int j = 1; j < 4; j++) {
                    orc_apply(hv, e, dir, apow + (j - 1) * P, hv_t, 1);
                    for (int64_t p = 0; p < P; p++) apow[j * P + p] = -I * tau * hv_t[p];
                    orc_apply(hv, e, dir, bpow + (j - 1) * P, hv_t, 1);
                    for (int64_t p = 0; p < P; p++) bpow[j * P + p] = I * tau * hv_t[p];
                }
                cplx acc = 0.0;
                for (int n = 1; n <= 4; n++)
                    for (int j = 0; j < n; j++) {
                        const cplx *bj = bpow + j * P;
                        const cplx *am = apow + (n - 1 - j) * P;
                        cplx ip = 0.0;
                        for (int64_t p = 0; p < P; p++) ip += conj(bj[p]) * X[p] * am[p];
                        acc += invfact[n] * (-I * tau) * h3 * ip;
                    }
                g += 2.0 * creal(acc);
            }
            grad[k] = g;
            memcpy(chi, chis, vb); /* chi_k = chi'_0 */
        }
    }
    free(ck); free(psi); free(tmp); free(chi); free(seg); free(psis);
    free(chis); free(apow); free(bpow); free(hv_t); free(X);
    return J;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
