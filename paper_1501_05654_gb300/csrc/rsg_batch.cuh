// Per-system stencil arguments of the batched kernels: the ApplyArgs view of
// one system of a batch (Horner stage: out = alpha * H in + base, base = the
// caller's state block, no field, projector terms added by the batched
// scatter).
#pragma once

#include "rsg_internal.h"

namespace rsg {

__device__ __forceinline__ ApplyArgs<float> batch_args(const SysArgs &S, int in_c, int out_c, float ar,
                                                       float ai) {
    ApplyArgs<float> a;
    a.in = S.vec[in_c];
    a.out = S.vec[out_c];
    a.base = S.vec[0];
    a.acc = nullptr;
    a.acc_base = nullptr;
    a.rows = S.rows;
    a.tiles = S.tiles;
    a.nx = S.nx;
    a.ny = S.ny;
    a.nz = S.nz;
    a.SV = S.SV;
    a.V = S.V;
    a.f0 = a.fx = a.fy = a.fz = 0.f;
    for (int k = 0; k < 5; k++) a.w[k] = S.w[k];
    a.ar = ar;
    a.ai = ai;
    a.br = 1.f;
    a.bi = 0.f;
    a.gr = a.gi = 0.f;
    a.nl_ptr = nullptr;
    a.nl_ent = nullptr;
    a.q_atom = nullptr;
    a.q_p = nullptr;
    a.D = nullptr;
    a.npmax = 0;
    a.P = S.P;
    a.err = nullptr;
    return a;
}

}  // namespace rsg
