// Device helpers shared by the apply kernels (apply_unit.cu: sum
// factorisation in registers; apply_cellmat.cu: cell matrices on the tensor
// cores; apply.cu: the p >= 3 plane kernel): the patch-node table of the
// packed-unit kernels and the 16-byte scatter-add into Y.
#pragma once

#include "fe_internal.h"

namespace femf {
namespace {

// 16-byte chunk of one block row added into Y
__device__ __forceinline__ void red_chunk(float* dst, const float* v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(dst), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]) : "memory");
}
__device__ __forceinline__ void red_chunk(double* dst, const double* v) {
    if (v[0] != 0.0) atomicAdd(dst, v[0]);
    if (v[1] != 0.0) atomicAdd(dst + 1, v[1]);
}

// Node `node` of the (2p+1)^3 patch (px, py, pz): (slot << 16) | row, slot
// b = dx + 2 dy + 4 dz naming the row block that owns the node (patch
// (px - 1 + dx, py - 1 + dy, pz - 1 + dz)) and row its position there; -1 for a
// Dirichlet boundary node.
template <int P>
__device__ __forceinline__ int node_entry(int node, int px, int py, int pz, int lx, int ly, int lz, int dirichlet) {
    constexpr int Q = 2 * P, NP = 2 * P + 1;
    const int i = node % NP, j = (node / NP) % NP, k = node / (NP * NP);
    const int I = Q * px + i, J = Q * py + j, K = Q * pz + k;
    if (dirichlet && (I == 0 || J == 0 || K == 0 || I == lx - 1 || J == ly - 1 || K == lz - 1)) return -1;
    const int dx = (i == 0 && px > 0) ? 0 : 1;
    const int dy = (j == 0 && py > 0) ? 0 : 1;
    const int dz = (k == 0 && pz > 0) ? 0 : 1;
    const int ii = dx ? i : Q, jj = dy ? j : Q, kk = dz ? k : Q;
    const int qx = px - 1 + dx, qy = py - 1 + dy, qz = pz - 1 + dz;
    const int nxq = Q + (qx == 0), nyq = Q + (qy == 0);
    const int row = (ii - (qx != 0)) + nxq * ((jj - (qy != 0)) + nyq * (kk - (qz != 0)));
    return ((dx + 2 * dy + 4 * dz) << 16) | row;
}

}  // namespace
}  // namespace femf
