// Antisymmetric-image boundary of a box mesh (rsg_mesh_set_boundary with
// RSG_BC_ODD).  The walls sit one spacing outside the mesh, at bounding-box
// index -1 and n along each axis.  A stencil neighbour outside the mesh
// takes the value of its mirror image about the wall, with the sign flipped
// once per reflection, and a neighbour on a wall is zero.  With these ghosts
// minus the discrete Laplacian of a box has the closed-form eigenvalues
// sum_d sigma(pi m_d / (n_d + 1)) / h^2 (sigma the symbol of the stencil,
// eigenvectors products of sines), so box eigenvalues converge at the
// stencil's order; with zero ghosts they converge at first order only.
#pragma once

#include "rsg_internal.h"
#include "rsg_vec.cuh"

namespace rsg {

// Reflects index i of an axis with n points into [0, n); false on a wall or
// when one reflection does not reach the mesh.
__device__ __forceinline__ bool odd_reflect(int &i, int n, bool &neg) {
    if (i < 0) {
        i = -2 - i;
        neg = !neg;
    } else if (i >= n) {
        i = 2 * n - i;
        neg = !neg;
    }
    return i >= 0 && i < n;
}

// Vector v of bounding-box site (x, y, z) under the image rule.
template <typename R>
__device__ __forceinline__ typename VT<R>::T odd_site(const typename VT<R>::T *in, const Row *rows, int x, int y,
                                                      int z, int nx, int ny, int nz, int SV, int v) {
    bool neg = false;
    if (!odd_reflect(x, nx, neg) || !odd_reflect(y, ny, neg) || !odd_reflect(z, nz, neg)) return VT<R>::zero();
    const Row rw = rows[(int64_t)z * ny + y];
    if (x < rw.xmin || x > rw.xmax) return VT<R>::zero();
    const typename VT<R>::T u = VT<R>::ldg(in + ((int64_t)rw.start + (x - rw.xmin)) * SV + v);
    return neg ? VT<R>::scale((R)-1, u) : u;
}

}  // namespace rsg
