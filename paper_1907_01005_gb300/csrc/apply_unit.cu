// Register-resident matrix-free apply for p <= 2 (Alg. 6 restricted to the
// source pattern).
//
// One CTA processes one packed work unit: a patch and up to four of its
// column blocks (at most 32 columns, "lanes").  A thread owns one cell and
// one lane: it holds all (p+1)^3 nodal values of its cell-column in
// registers and applies the whole sum-factorised cell operator there --
// interpolation to the Gauss points along x, y, z, the quadrature (three 1D
// Laplacian sweeps and the potential) and the transposed interpolation.
//
// Data movement works on 16-byte row chunks (block rows are padded to 16
// bytes): the gather is a set of asynchronous 16-byte copies (cp.async, zero
// fill for absent blocks and boundary nodes) into a patch tensor
// U[node][kUnitLdSum] whose rows hold the unit's blocks side by side (the 32
// lanes of a warp then read one row: no bank conflicts between blocks, and
// the row stride is a compile-time constant); the cells' results are summed
// into a matching zeroed tensor in a fixed order (merge_cells_store, no
// shared-memory atomics); the tensor goes
// into Y in the ordered, conflict-free write of unit_common.cuh (units in
// descending patch rank, first writer stores, later contributors add), so Y
// needs no zero-fill and no global atomics are used.
#include <algorithm>

#include "fe_internal.h"
#include "unit_common.cuh"

namespace femf {
namespace {

template <typename T, int P>
struct UnitGeo {
    static constexpr int N = P + 1, NP = 2 * P + 1, NPN = NP * NP * NP, N3 = N * N * N;
    static constexpr int L = kUnitLanes;             // columns of a unit, one per thread of a cell
    static constexpr int THREADS = 8 * L;
    static constexpr int CH = 16 / sizeof(T);          // elements per 16-byte chunk
    static constexpr int TEN = NPN * kUnitLdSum;       // elements of one patch tensor (all blocks)
    // the region of U also holds the exchange buffer of the cell merge
    static constexpr int UEX = TEN > 2 * kMergeFace<P> ? TEN : 2 * kMergeFace<P>;
    // gathered input U, accumulated output Yp, V at the Gauss points
    static constexpr size_t bytes = (size_t)(UEX + TEN + 8 * N3) * sizeof(T);
    static_assert(UEX * sizeof(T) % 16 == 0, "the patch tensors start on 16-byte boundaries");
};

// resident CTAs per SM the register budget must allow (a cell-column's
// values and their sweep partner take 2 (p+1)^3 registers)
template <typename T>
constexpr int kUnitMinBlocks = sizeof(T) == 4 ? 4 : 2;

template <typename T, int P, bool MASS>
__global__ void __launch_bounds__(UnitGeo<T, P>::THREADS, kUnitMinBlocks<T>)
    apply_unit_kernel(const ApplyUnitArgs<T> a) {
    using G = UnitGeo<T, P>;
    constexpr int N = G::N, NP = G::NP, NPN = G::NPN, N3 = G::N3, L = G::L;
    constexpr int CH = G::CH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* U = reinterpret_cast<T*>(smem_raw);         // [NPN][kUnitLdSum]: block b at columns sBase[b] ..
    T* Yp = U + G::UEX;                            // same layout, accumulated cell results
    T* Vs = Yp + G::TEN;                           // [8][N3]  V at the Gauss points
    __shared__ int32_t sOff[kUnitBlocks][8], sHout[kUnitBlocks][8], sHin[kUnitBlocks][8];
    __shared__ int sHn[kUnitBlocks][8], sHb[kUnitBlocks][8];   // fetched halo slots: elements, buffer offsets
    __shared__ int sLaneB[L], sLaneA[L], sMask[kUnitBlocks], sBase[kUnitBlocks], sLd[kUnitBlocks];
    __shared__ int sNode[NPN];                     // node_entry: row, owner slot, first-writer and boundary bits
    __shared__ int sOwn[NPN];                      // own_row_entry of the patch's own rows
    __shared__ __align__(16) Unit sUnit[2];        // the unit's record and the next one's
    __shared__ int64_t sItem, sNext;
    const int tid = threadIdx.x;
    constexpr int kElem16 = 16 / sizeof(T);        // elements per 16-byte offset unit
    // a unit record into sUnit[buf]: 16-byte asynchronous copies
    static_assert(sizeof(Unit) % 16 == 0, "unit records are whole 16-byte chunks");
    auto fetch_unit = [&](int64_t ticket_, int buf) {
        if (tid < (int)(sizeof(Unit) / 16)) {
            const char* src = reinterpret_cast<const char*>(a.units + (a.n_units - 1 - ticket_)) + 16 * tid;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&sUnit[buf]) + 16u * tid;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
        }
    };
    // Units are taken from a work counter in descending order (descending
    // patch rank, the order of the write): one per CTA, or (persistent
    // launch) until the list is exhausted.  A persistent CTA takes its next
    // ticket as a unit starts and copies the next record in after the cell
    // work, so neither round trip delays the next unit.
    if (tid == 0) sItem = (int64_t)atomicAdd(a.ticket, 1ull);
    __syncthreads();
    int64_t ticket = sItem;
    int cur = 0;
    if (ticket < a.n_units) fetch_unit(ticket, 0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    unsigned long long next_raw = 0ull;            // thread 0: the next ticket
    while (ticket < a.n_units) {
    const int64_t item = a.n_units - 1 - ticket;
    const Unit& unit = sUnit[cur];
    if (a.persistent && tid == 0) next_raw = atomicAdd(a.ticket, 1ull);
    bool prefetched = false;
    const int px = unit.pxyz & 1023, py = (unit.pxyz >> 10) & 1023, pz = unit.pxyz >> 20;
    // Work-list check: the host packs 1..kUnitBlocks blocks with 1 <= width <= ld,
    // ld a whole number of 16-byte chunks, at most L lanes and sum(ld) <= kUnitLdSum.
    // A unit that breaks this would overrun shared memory: it sets the status
    // word and is skipped (the same decision in every thread of the CTA).
    bool unit_ok = unit.nb >= 1 && unit.nb <= kUnitBlocks;
    if (unit_ok) {
        int lds = 0, lanes = 0;
        for (int q = 0; q < unit.nb; ++q) {
            const int wq = unit.width[q], lq = unit.ld[q];
            unit_ok = unit_ok && wq >= 1 && wq <= lq && lq % CH == 0;
            lds += lq;
            lanes += wq;
        }
        unit_ok = unit_ok && lds <= kUnitLdSum && lanes <= L;
    }
    const bool in_mesh = px < a.npx && py < a.npy && pz < a.npz;
    unit_ok = unit_ok && in_mesh;
    if (!unit_ok && tid == 0) atomicExch(a.status, kDevBadTile);
    if (unit_ok) {

    // ---- unit tables --------------------------------------------------------
    if (tid < L) {
        int b = -1, col = 0, pref = 0;
        for (int q = 0; q < unit.nb; ++q) {
            const int wq = unit.width[q];
            if (tid >= pref && tid < pref + wq) { b = q; col = tid - pref; }
            pref += wq;
        }
        sLaneB[tid] = b;
        sLaneA[tid] = col;
        const bool has = (tid >> 3) < unit.nb;
        sOff[tid >> 3][tid & 7] = has ? unit.off[tid >> 3][tid & 7] : -1;
        sHout[tid >> 3][tid & 7] = has ? unit.hout[tid >> 3][tid & 7] : -1;
        sHin[tid >> 3][tid & 7] = has ? unit.hin[tid >> 3][tid & 7] : -1;
        // elements of the halo slots (b, e) this unit fetches for its own rows
        const int hb = tid >> 3, he = tid & 7;
        sHn[hb][he] = (he > 0 && has && unit.off[hb][7] >= 0 && unit.hin[hb][he] >= 0)
                          ? halo_slot_rows<P>(he, px, py, pz) * unit.ld[hb] : 0;
    }
    if (tid == 0) {
        int base = 0;
        for (int q = 0; q < kUnitBlocks; ++q) {
            const int ldq = q < unit.nb ? unit.ld[q] : 0;
            sBase[q] = base;                       // first column of block q in a node row
            sLd[q] = ldq;
            sMask[q] = q < unit.nb ? unit.cellmask[q] : 0;
            base += ldq;
        }
    }
    for (int n = tid; n < NPN; n += blockDim.x)
        sNode[n] = node_entry<P>(n, px, py, pz, a.lx, a.ly, a.lz, a.dirichlet, a.npx, a.npy, a.npz);
    // own-row table for the store, by the threads past the node table
    for (int r = tid - NPN; r >= 0 && r < own_rows_of<P>(px, py, pz); r += blockDim.x - NPN)
        sOwn[r] = own_row_entry<P>(r, px, py, pz);
    __syncthreads();

    static_assert(kUnitBlocks == 4, "task index: node << 2 | block");
    const int nb = unit.nb;
    constexpr int S = kUnitLdSum;                  // node row: the unit's blocks side by side
    // ---- gather: asynchronous 16-byte copies of block rows ------------------
    // one task per (node, block): the row's table lookups once, then its
    // 16-byte chunks
    {
        const unsigned ubase = (unsigned)__cvta_generic_to_shared(U);
        for (int e = tid; e < NPN * kUnitBlocks; e += blockDim.x) {
            const int node = e >> 2, b = e & 3;
            if (b >= nb) continue;
            const int ld = sLd[b];
            const int ne = sNode[node];
            const int32_t o = (ne & kBoundary) ? -1 : sOff[b][(ne >> 16) & 7];
            const bool ok = o >= 0;
            const T* src = ok ? a.P + (int64_t)o * kElem16 + (ne & 0xffff) * ld : a.P;
            const unsigned dst = ubase + (unsigned)((node * S + sBase[b]) * sizeof(T));
            for (int c0 = 0; c0 < ld; c0 += CH)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + c0 * (int)sizeof(T)),
                             "l"(ok ? src + c0 : src), "r"(ok ? 16 : 0) : "memory");
        }
        // the potential of the patch's cells (contiguous, 16-byte aligned)
        if constexpr (!MASS) {
            const T* Vg = a.Vq + (int64_t)unit.patch * 8 * N3;
            const unsigned vbase = (unsigned)__cvta_generic_to_shared(Vs);
            for (int e = tid; e < 8 * N3 / CH; e += blockDim.x)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(vbase + 16u * e), "l"(Vg + e * CH)
                             : "memory");
        }
        // zero the output tensor while the copies are in flight
        const int ten4 = NPN * S / CH;
        for (int e = tid; e < ten4; e += blockDim.x) reinterpret_cast<uint4*>(Yp)[e] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();

    // ---- cell operator in registers -----------------------------------------
    {
        const int cell = tid / L, lane = tid % L;
        const int cx = cell & 1, cy = (cell >> 1) & 1, cz = (cell >> 2) & 1;
        const int b = sLaneB[lane];
        const bool act = b >= 0 && ((sMask[b] >> cell) & 1);
        // element of local node (z, y, x) of this cell in both patch tensors
        const int base = b >= 0 ? sBase[b] + sLaneA[lane] + ((cz * P * NP + cy * P) * NP + cx * P) * S : 0;
        T u[N][N][N], t[N][N][N];
        if (act) {
#pragma unroll
            for (int z = 0; z < N; ++z)
#pragma unroll
                for (int y = 0; y < N; ++y)
#pragma unroll
                    for (int x = 0; x < N; ++x) u[z][y][x] = U[base + ((z * NP + y) * NP + x) * S];
        }
        __syncthreads();                               // U is read: it becomes the merge's exchange buffer
        if (act) {
            const auto& K = a.k;
            // Sweeps run coefficient-outer: each coefficient is applied to all
            // N^2 lines of the sweep.
#define SWEEP(C, IDX_D, IDX_S)                                               \
    _Pragma("unroll") for (int q = 0; q < N; ++q) {                          \
        _Pragma("unroll") for (int p2 = 0; p2 < N; ++p2) {                   \
            const T c = C[q][p2];                                            \
            _Pragma("unroll") for (int m = 0; m < N; ++m)                    \
            _Pragma("unroll") for (int n = 0; n < N; ++n) {                  \
                T& d = IDX_D;                                                \
                d = fma(c, IDX_S, p2 == 0 ? T(0) : d);                       \
            }                                                                \
        }                                                                    \
    }
            // interpolate to the Gauss points along x, y, z
            SWEEP(K.S, t[m][n][q], u[m][n][p2])
            SWEEP(K.S, u[m][q][n], t[m][p2][n])
            SWEEP(K.S, t[q][m][n], u[p2][m][n])
            // quadrature: V u_q plus the three collocation Laplacian sweeps
            // (|J| is folded into the coefficients: A / |J| here, |J| Sb in the
            // first transposed sweep below); the mass operator keeps u_q
            const T* Vc = Vs + cell * N3;
#pragma unroll
            for (int z = 0; z < N; ++z)
#pragma unroll
                for (int y = 0; y < N; ++y)
#pragma unroll
                    for (int x = 0; x < N; ++x) u[z][y][x] = MASS ? t[z][y][x] : Vc[(z * N + y) * N + x] * t[z][y][x];
#pragma unroll
            for (int q = 0; q < (MASS ? 0 : N); ++q)
#pragma unroll
                for (int l = 0; l < N; ++l) {
                    const T c0 = K.A[0][q][l], c1 = K.A[1][q][l], c2 = K.A[2][q][l];
#pragma unroll
                    for (int m = 0; m < N; ++m)
#pragma unroll
                        for (int n = 0; n < N; ++n) {
                            u[m][n][q] = fma(c0, t[m][n][l], u[m][n][q]);
                            u[m][q][n] = fma(c1, t[m][l][n], u[m][q][n]);
                            u[q][m][n] = fma(c2, t[l][m][n], u[q][m][n]);
                        }
                }
            // integrate: transposed interpolation along x (with |J|), y, z
            SWEEP(K.Sb1, t[m][n][q], u[m][n][p2])
            SWEEP(K.Sb, u[m][q][n], t[m][p2][n])
            SWEEP(K.Sb, t[q][m][n], u[p2][m][n])
#undef SWEEP
        } else {
#pragma unroll
            for (int z = 0; z < N; ++z)
#pragma unroll
                for (int y = 0; y < N; ++y)
#pragma unroll
                    for (int x = 0; x < N; ++x) t[z][y][x] = T(0);
        }
        // the cells' results into the patch tensor: nodes on faces, edges and
        // the centre are shared with the neighbouring cells and are summed in
        // a fixed order, each node stored once
        merge_cells_store<P, S, NP, false>(t, cell, lane, b >= 0, U, Yp, base);
    }
    if (a.persistent && tid == 0) sNext = (int64_t)next_raw;
    __syncthreads();
    if (a.persistent) {                                // the next record, while this unit writes
        if (sNext < a.n_units) fetch_unit(sNext, cur ^ 1);
        prefetched = true;
    }

    // ---- write into Y (Alg. 6, write step; unit_common.cuh) ------------------
    // (1) contributions to the lower neighbours' rows into their halo slots
    for (int e = tid; e < NPN * kUnitBlocks; e += blockDim.x) {
        const int node = e >> 2, b = e & 3;
        if (b >= nb) continue;
        const int ne = sNode[node];
        const int slot = (ne >> 16) & 7;
        if (slot == 7 || (ne & kBoundary)) continue;
        const int32_t h = sHout[b][slot];
        if (h < 0) continue;
        const int ld = sLd[b];
        put_halo_row(a.halo + (int64_t)h * kElem16 + (ne >> kAuxShift) * ld, Yp + node * S + sBase[b], ld);
    }
    __syncthreads();
    // the patch is marked by warp 1 while warp 0 waits for the neighbours
    if (tid == 32) mark_done(a.done, px + a.npx * (py + a.npy * pz));
    // (2) the upper neighbours' halos addressed to this patch, fetched into
    // the free gather buffer in one round of asynchronous copies (the
    // barrier in fetch_halo holds the other warps until warp 0 is through)
    if (tid < 32 && !wait_upper_neighbours(a.done, a.count, px, py, pz, a.npx, a.npy, a.npz) && tid == 0)
        atomicExch(a.status, kDevTimeout);
    fetch_halo(U, a.halo, sHin, sHn, sHb, nb);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // (3) own rows: own part plus the halo rows, stored once
    store_own_rows<P>(
        [&](int b) -> T* { return sOff[b][7] >= 0 ? a.Y + (int64_t)sOff[b][7] * kElem16 : nullptr; }, Yp, S, sBase,
        sLd, U, sHb, sHn, sNode, sOwn, nb, px, py, pz);
    }  // unit_ok
    else if (tid == 0 && in_mesh) {
        mark_done(a.done, px + a.npx * (py + a.npy * pz));   // a skipped unit: nobody waits for it
    }
    if (a.persistent && !prefetched) {                 // a skipped unit: the next record now
        if (tid == 0) sNext = (int64_t)next_raw;
        __syncthreads();
        if (sNext < a.n_units) fetch_unit(sNext, cur ^ 1);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();                                   // the unit's rows are written (shared tables free)
    if (!a.persistent) break;
    ticket = sNext;
    cur ^= 1;
    }
}

template <typename T, int P, bool MASS>
cudaError_t unit_attrs() {
    using G = UnitGeo<T, P>;
    cudaError_t e = cudaFuncSetAttribute(apply_unit_kernel<T, P, MASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(apply_unit_kernel<T, P, MASS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

template <typename T, int P>
cudaError_t launch_units_p(const ApplyUnitArgs<T>& a, cudaStream_t s) {
    using G = UnitGeo<T, P>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = unit_attrs<T, P, false>();
        if (e == cudaSuccess) e = unit_attrs<T, P, true>();
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (a.n_units == 0) return cudaSuccess;
    unsigned grid = (unsigned)a.n_units;
    if (a.persistent) {
        const int sms = usable_sms(a.sm_limit);
        if (sms < 1) return cudaErrorInvalidDevice;
        grid = (unsigned)std::min<int64_t>(a.n_units, (int64_t)sms * std::max(1, a.ctas_per_sm));
    }
    if (a.mass)
        apply_unit_kernel<T, P, true><<<grid, G::THREADS, G::bytes, s>>>(a);
    else
        apply_unit_kernel<T, P, false><<<grid, G::THREADS, G::bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_apply_units(int p, const ApplyUnitArgs<T>& a, cudaStream_t s) {
    switch (p) {
        case 1: return launch_units_p<T, 1>(a, s);
        case 2: return launch_units_p<T, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_apply_units<float>(int, const ApplyUnitArgs<float>&, cudaStream_t);
template cudaError_t launch_apply_units<double>(int, const ApplyUnitArgs<double>&, cudaStream_t);

}  // namespace femf
