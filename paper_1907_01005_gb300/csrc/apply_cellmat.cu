// Cell-matrix form of the apply for p <= 2, FP32, on the tcgen05 tensor cores.
//
// The element view of the operator (Sec. 3.2, Eq. fe_matrices_cell_based):
// H = sum_K P_K^T H_K P_K, with the element matrices applied as dense
// products on the element level (the "FE op. (BCSR gemm)" flavour of Sec. 4.2).
// On the box meshes here every cell has the same affine geometry, so
//   H_K u = K_L u + Sb3 (|J| V_K o (S3 u)),
// with three matrices shared by all cells: K_L = Sb3 L_c S3 (kinetic part,
// L_c the collocation Laplacian at the Gauss points), S3 = S x S x S
// (interpolation to the Gauss points) and Sb3 (its weighted transpose); only
// the potential V_K at the cell's Gauss points differs between cells.  The
// mass operator is M_K u = (|J| Sb3 S3) u.
//
// Work decomposition: the packed work units of the register kernel (a patch
// and up to 32 columns of its column blocks).  Thread (cell, lane) owns row
// m = 32 cell + lane of the operand A[m][k] = u of its cell-column at cell
// node k, so the unit is two 128-row tiles.  Per tile:
//   stage 1  D[:, 0:npad]      = A K_L^T,  D[:, npad:2 npad] = A S3^T   (N = 2 npad)
//   stage 2  D[:, 0:npad]     += (|J| V o D[:, npad:2 npad]) Sb3^T     (N = npad)
// as tcgen05.mma kind::tf32 with the accumulators in tensor memory.  FP32
// accuracy comes from a 3-term TF32 split of both operands,
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi   (a_hi = TF32 rounding of a),
// which leaves an error of about 2^-21 relative per product.
//
// Data movement is that of the register kernel: 16-byte cp.async gather of the
// patch tensor (node rows of kUnitLdSum with the unit's blocks side by side),
// the cells' results summed into a zeroed patch tensor in a fixed order
// (merge_cells_store; here the tensor reuses the gather buffer and the
// exchange uses the free A tiles), and the conflict-free write into Y of
// unit_common.cuh (units in descending patch rank, halo slots).  The constant operand
// tiles (both parts of K_L, S3, Sb3) are copied once per CTA; CTAs are
// persistent and take units from a work counter.
#include <algorithm>
#include <cstdint>

#include "fe_internal.h"
#include "tc_common.cuh"
#include "unit_common.cuh"

namespace femf {
namespace {

template <int P>
struct CmGeo {
    static constexpr int N = P + 1, NP = 2 * P + 1, NPN = NP * NP * NP, N3 = N * N * N;
    static constexpr int NPAD = cellmat_npad(P);   // cell nodes padded: MMA N of one matrix
    static constexpr int KSTEPS = (N3 + 7) / 8;    // K = 8 per TF32 MMA
    static constexpr int L = kUnitLanes;
    static constexpr int THREADS = 8 * L;          // one A row per thread: 2 tiles of 128
    static constexpr int CH = 4;                   // floats per 16-byte chunk
    static constexpr int TEN = NPN * kUnitLdSum;   // floats of the patch tensor
    static constexpr int TILE = 128 * 128;         // bytes of a 128-row operand tile (rows of 32 floats)
    // dynamic shared memory, from a 1024-byte aligned base (the period of the
    // 128-byte swizzle): A high parts (2 tiles), A low parts, the constant
    // set (B1 high/low: 2 npad rows each; B2 high/low: npad rows each), the
    // patch tensor, V at the Gauss points of the 8 cells
    static constexpr int OFF_AH = 0;
    static constexpr int OFF_AL = 2 * TILE;
    static constexpr int OFF_B1H = 4 * TILE;
    static constexpr int OFF_B1L = OFF_B1H + 2 * NPAD * 128;
    static constexpr int OFF_B2H = OFF_B1L + 2 * NPAD * 128;
    static constexpr int OFF_B2L = OFF_B2H + NPAD * 128;
    static constexpr int OFF_U = OFF_B2L + NPAD * 128;
    static constexpr int OFF_V = OFF_U + TEN * 4;
    static constexpr int bytes = OFF_V + 8 * N3 * 4 + 1024;   // + alignment slack
    static constexpr int TMEM_COLS = 4 * NPAD;                 // 2 tiles x 2 npad FP32 columns
    static constexpr int SET_FLOATS = cellmat_set_floats(P);
    static_assert(OFF_B1H % 1024 == 0 && OFF_B1L % 1024 == 0 && OFF_B2H % 1024 == 0 && OFF_B2L % 1024 == 0,
                  "operand tiles must start on the swizzle period");
    static_assert((OFF_B2L + NPAD * 128 - OFF_B1H) == cellmat_set_floats(P) * 4, "constant set size");
    static_assert(OFF_U % 16 == 0 && OFF_V % 16 == 0, "16-byte copies");
    static_assert(TMEM_COLS == 64 || TMEM_COLS == 128, "tensor-memory allocation: power of two >= 32");
};

// Row r of a 128-row tile pair (high parts at hi, low parts at lo): values
// x[0 .. 4 nch - 1] as 16-byte chunks, chunk c stored at chunk c ^ (r & 7).
template <int NCH>
__device__ __forceinline__ void store_row_split(unsigned char* hi, unsigned char* lo, int r, const float* x) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        float h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = tf32_hi(x[4 * c + q]);
            l[q] = x[4 * c + q] - h[q];
        }
        const int o = r * 128 + ((c ^ (r & 7)) << 4);
        *reinterpret_cast<float4*>(hi + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(lo + o) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;   // 0.2 s for a few microseconds of MMA work

template <int P, bool MASS>
__global__ void __launch_bounds__(CmGeo<P>::THREADS, 2) apply_cellmat_kernel(const CellMatArgs a) {
    using G = CmGeo<P>;
    constexpr int N = G::N, NP = G::NP, NPN = G::NPN, N3 = G::N3, L = G::L, NPAD = G::NPAD;
    constexpr int CH = G::CH, KSTEPS = G::KSTEPS, KCH = (8 * KSTEPS) / 4;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    unsigned char* sm = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
    float* U = reinterpret_cast<float*>(sm + G::OFF_U);    // gathered patch tensor, then the cells' results
    float* Vs = reinterpret_cast<float*>(sm + G::OFF_V);   // [8][N3]
    __shared__ int32_t sOff[kUnitBlocks][8], sHout[kUnitBlocks][8], sHin[kUnitBlocks][8];
    __shared__ int sHn[kUnitBlocks][8], sHb[kUnitBlocks][8];   // fetched halo slots: elements, buffer offsets
    __shared__ int sLaneB[L], sLaneA[L], sMask[kUnitBlocks], sBase[kUnitBlocks], sLd[kUnitBlocks];
    __shared__ int sNode[NPN];
    __shared__ int64_t sItem;
    __shared__ __align__(8) uint64_t sBar;
    __shared__ uint32_t sTmem;
    __shared__ int sFail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar = smem_u32(&sBar);

    // ---- constant operand tiles (pre-swizzled), tensor memory, barrier ------
    {
        const unsigned dst = smem_u32(sm + G::OFF_B1H);
        for (int e = tid; e < G::SET_FLOATS / 4; e += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * e), "l"(a.consts + 4 * e)
                         : "memory");
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        fence_async_smem();                               // the tiles feed the tensor cores
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTmem)),
                     "r"(G::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sFail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sTmem;
    uint32_t phase = 0;

    // row of this thread: tile t, row r; its accumulators in tensor memory
    const int t = tid >> 7, r = tid & 127;
    unsigned char* aHi = sm + G::OFF_AH + t * G::TILE;
    unsigned char* aLo = sm + G::OFF_AL + t * G::TILE;
    const uint32_t tD = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(t * 2 * NPAD);
    const int cell = tid / L, lane = tid % L;
    const int cx = cell & 1, cy = (cell >> 1) & 1, cz = (cell >> 2) & 1;

    if (tid == 0) sItem = (int64_t)atomicAdd(a.ticket, 1ull);
    __syncthreads();
    int64_t ticket = sItem;
    while (ticket < a.n_units) {
        // units in descending order: descending patch rank, the order of the write
        const Unit& unit = a.units[a.n_units - 1 - ticket];
        const int px = unit.pxyz & 1023, py = (unit.pxyz >> 10) & 1023, pz = unit.pxyz >> 20;
        const bool in_mesh = px < a.npx && py < a.npy && pz < a.npz;
        // work-list check, as in the register kernel
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
        unit_ok = unit_ok && in_mesh;
        if (!unit_ok && tid == 0) atomicExch(a.status, kDevBadTile);
        if (unit_ok) {
            // ---- unit tables ------------------------------------------------
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
            }
            if (tid == 0) {
                int base = 0;
                for (int q = 0; q < kUnitBlocks; ++q) {
                    const int ldq = q < unit.nb ? unit.ld[q] : 0;
                    sBase[q] = base;                   // first column of block q in a node row
                    sLd[q] = ldq;
                    sMask[q] = q < unit.nb ? unit.cellmask[q] : 0;
                    base += ldq;
                }
            }
            for (int n = tid; n < NPN; n += blockDim.x)
                sNode[n] = node_entry<P>(n, px, py, pz, a.lx, a.ly, a.lz, a.dirichlet, a.npx, a.npy, a.npz);
            __syncthreads();

            static_assert(kUnitBlocks == 4, "task index: node << 2 | block");
            const int nb = unit.nb;
            constexpr int S = kUnitLdSum;                 // node row: the unit's blocks side by side
            // ---- gather: one task per (node, block) row ----------------------
            {
                const unsigned ubase = smem_u32(U);
                for (int e = tid; e < NPN * kUnitBlocks; e += blockDim.x) {
                    const int node = e >> 2, b = e & 3;
                    if (b >= nb) continue;
                    const int ld = sLd[b];
                    const int ne = sNode[node];
                    const int32_t o = (ne & kBoundary) ? -1 : sOff[b][(ne >> 16) & 7];
                    const bool ok = o >= 0;
                    const float* src = ok ? a.P + (int64_t)o * 4 + (ne & 0xffff) * ld : a.P;
                    const unsigned dst = ubase + (unsigned)((node * S + sBase[b]) * 4);
                    for (int c0 = 0; c0 < ld; c0 += CH)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + 4 * c0),
                                     "l"(ok ? src + c0 : src), "r"(ok ? 16 : 0) : "memory");
                }
                if constexpr (!MASS) {
                    const float* Vg = a.Vq + (int64_t)unit.patch * 8 * N3;
                    const unsigned vbase = smem_u32(Vs);
                    for (int e = tid; e < 8 * N3 / CH; e += blockDim.x)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(vbase + 16u * e),
                                     "l"(Vg + e * CH)
                                     : "memory");
                }
                asm volatile("cp.async.wait_all;\n" ::: "memory");
            }
            __syncthreads();

            // ---- stage 1 operand: the thread's cell-column at its cell's nodes
            const int b = sLaneB[lane];
            const bool act = b >= 0 && ((sMask[b] >> cell) & 1);
            const int base = b >= 0 ? sBase[b] + sLaneA[lane] + ((cz * P * NP + cy * P) * NP + cx * P) * S : 0;
            {
                float x[4 * KCH];
#pragma unroll
                for (int k = 0; k < 4 * KCH; ++k) x[k] = 0.f;
                if (act) {
#pragma unroll
                    for (int z = 0; z < N; ++z)
#pragma unroll
                        for (int y = 0; y < N; ++y)
#pragma unroll
                            for (int xx = 0; xx < N; ++xx)
                                x[(z * N + y) * N + xx] = U[base + ((z * NP + y) * NP + xx) * S];
                }
                store_row_split<KCH>(aHi, aLo, r, x);
            }
            fence_async_smem();
            __syncthreads();                              // A complete; the patch tensor is free
            if (tid == 0) {
                tc_fence_after();
                const uint32_t id1 = tf32_idesc(128, MASS ? NPAD : 2 * NPAD);
#pragma unroll
                for (int tt = 0; tt < 2; ++tt) {
                    const uint32_t d = tmem + (uint32_t)(tt * 2 * NPAD);
                    const uint32_t ah = smem_u32(sm + G::OFF_AH + tt * G::TILE), al = smem_u32(sm + G::OFF_AL + tt * G::TILE);
                    const uint32_t bh = smem_u32(sm + G::OFF_B1H), bl = smem_u32(sm + G::OFF_B1L);
#pragma unroll
                    for (int kk = 0; kk < KSTEPS; ++kk) {
                        mma_tf32(d, sw128_desc(ah + 32 * kk), sw128_desc(bh + 32 * kk), id1, kk > 0);
                        mma_tf32(d, sw128_desc(ah + 32 * kk), sw128_desc(bl + 32 * kk), id1, 1);
                        mma_tf32(d, sw128_desc(al + 32 * kk), sw128_desc(bh + 32 * kk), id1, 1);
                    }
                }
                mma_commit(bar);
            }
            // zero the patch tensor for the results while the MMAs run
            const int ten4 = NPN * S / CH;
            for (int e = tid; e < ten4; e += blockDim.x) reinterpret_cast<uint4*>(U)[e] = make_uint4(0u, 0u, 0u, 0u);
            if (tid == 0 && !mbar_wait(bar, phase, kWaitLimitNs)) sFail = 1;
            phase ^= 1;
            __syncthreads();
            if (sFail) {                                  // count the unit as finished: no neighbour waits on it
                if (tid == 0) mark_done(a.done, px + a.npx * (py + a.npy * pz));
                break;
            }
            tc_fence_after();

            if constexpr (!MASS) {
                // ---- stage 2 operand: |J| V o u_q (|J| is in Sb3) -----------
                float uq[NPAD];
                tmem_load<NPAD>(tD + NPAD, uq);
                float x[4 * KCH];
#pragma unroll
                for (int k = 0; k < 4 * KCH; ++k) x[k] = k < N3 ? uq[k] * Vs[cell * N3 + k] : 0.f;
                store_row_split<KCH>(aHi, aLo, r, x);
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t id2 = tf32_idesc(128, NPAD);
#pragma unroll
                    for (int tt = 0; tt < 2; ++tt) {
                        const uint32_t d = tmem + (uint32_t)(tt * 2 * NPAD);
                        const uint32_t ah = smem_u32(sm + G::OFF_AH + tt * G::TILE), al = smem_u32(sm + G::OFF_AL + tt * G::TILE);
                        const uint32_t bh = smem_u32(sm + G::OFF_B2H), bl = smem_u32(sm + G::OFF_B2L);
#pragma unroll
                        for (int kk = 0; kk < KSTEPS; ++kk) {
                            mma_tf32(d, sw128_desc(ah + 32 * kk), sw128_desc(bh + 32 * kk), id2, 1);
                            mma_tf32(d, sw128_desc(ah + 32 * kk), sw128_desc(bl + 32 * kk), id2, 1);
                            mma_tf32(d, sw128_desc(al + 32 * kk), sw128_desc(bh + 32 * kk), id2, 1);
                        }
                    }
                    mma_commit(bar);
                    if (!mbar_wait(bar, phase, kWaitLimitNs)) sFail = 1;
                }
                phase ^= 1;
                __syncthreads();
                if (sFail) {
                    if (tid == 0) mark_done(a.done, px + a.npx * (py + a.npy * pz));
                    break;
                }
                tc_fence_after();
            }

            // ---- the cell's result into the patch tensor ---------------------
            // (shared nodes summed in a fixed order through the free A tiles,
            // each node stored once)
            {
                float y[NPAD];
                tmem_load<NPAD>(tD, y);
                float tcell[N][N][N];
#pragma unroll
                for (int z = 0; z < N; ++z)
#pragma unroll
                    for (int yy = 0; yy < N; ++yy)
#pragma unroll
                        for (int xx = 0; xx < N; ++xx) tcell[z][yy][xx] = act ? y[(z * N + yy) * N + xx] : 0.f;
                static_assert(2 * kMergeFace<P> * 4 <= 4 * G::TILE, "exchange buffer in the A tiles");
                merge_cells_store<P, S, NP, false>(tcell, cell, lane, sLaneB[lane] >= 0,
                                                   reinterpret_cast<float*>(sm + G::OFF_AH), U, base);
            }
            tc_fence_before();
            __syncthreads();

            // ---- write into Y (unit_common.cuh), one task per (node, block) row
            for (int e = tid; e < NPN * kUnitBlocks; e += blockDim.x) {
                const int node = e >> 2, bb = e & 3;
                if (bb >= nb) continue;
                const int ne = sNode[node];
                const int slot = (ne >> 16) & 7;
                if (slot == 7 || (ne & kBoundary)) continue;
                const int32_t h = sHout[bb][slot];
                if (h < 0) continue;
                const int ldb = sLd[bb];
                put_halo_row(a.halo + (int64_t)h * 4 + (ne >> kAuxShift) * ldb, U + node * S + sBase[bb], ldb);
            }
            __syncthreads();
            // the patch is marked by warp 1 while warp 0 waits for the neighbours
            if (tid == 32) mark_done(a.done, px + a.npx * (py + a.npy * pz));
            if (warp == 0 && !wait_upper_neighbours(a.done, a.count, px, py, pz, a.npx, a.npy, a.npz) && tid == 0)
                atomicExch(a.status, kDevTimeout);
            // the halos addressed to this unit, fetched into the free A tiles
            // (slot sizes by warp 0, whose lanes read them in the prefix of
            // fetch_halo; its barrier publishes them)
            if (tid < kUnitBlocks * 8) {
                const int bb = tid >> 3, e = tid & 7;
                sHn[bb][e] = (e > 0 && bb < nb && sOff[bb][7] >= 0 && sHin[bb][e] >= 0)
                                 ? halo_slot_rows<P>(e, px, py, pz) * sLd[bb] : 0;
            }
            float* hbuf = reinterpret_cast<float*>(sm + G::OFF_AH);
            fetch_halo(hbuf, a.halo, sHin, sHn, sHb, nb);
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncthreads();
            // own rows: own part plus the halo rows, stored once
            store_own_rows<P>(
                [&](int bb) -> float* { return sOff[bb][7] >= 0 ? a.Y + (int64_t)sOff[bb][7] * 4 : nullptr; }, U, S,
                sBase, sLd, hbuf, sHb, sHn, sNode, nullptr, nb, px, py, pz);
        }  // unit_ok
        else if (tid == 0 && in_mesh) {
            mark_done(a.done, px + a.npx * (py + a.npy * pz));   // a skipped unit: nobody waits for it
        }
        __syncthreads();                                  // rows written; shared tables are rebuilt for the next unit
        if (tid == 0) sItem = (int64_t)atomicAdd(a.ticket, 1ull);
        __syncthreads();
        ticket = sItem;
    }

    // ---- teardown: on a time-out, give the MMAs in flight one more bounded
    // wait; then release the tensor memory ----------------------------------
    if (sFail) {
        if (tid == 0) {
            atomicExch(a.status, kDevTimeout);
            mbar_wait(bar, phase ^ 1, kWaitLimitNs);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS)
                     : "memory");
    }
}

template <int P>
cudaError_t launch_cellmat_p(const CellMatArgs& a, cudaStream_t s) {
    using G = CmGeo<P>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(apply_cellmat_kernel<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(apply_cellmat_kernel<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (a.n_units == 0) return cudaSuccess;
    const int sms = usable_sms(a.sm_limit);
    if (sms < 1) return cudaErrorInvalidDevice;
    const unsigned grid = (unsigned)std::min<int64_t>(a.n_units, (int64_t)sms * 2);
    if (a.mass)
        apply_cellmat_kernel<P, true><<<grid, G::THREADS, G::bytes, s>>>(a);
    else
        apply_cellmat_kernel<P, false><<<grid, G::THREADS, G::bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_cellmat(int p, const CellMatArgs& a, cudaStream_t s) {
    switch (p) {
        case 1: return launch_cellmat_p<1>(a, s);
        case 2: return launch_cellmat_p<2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace femf
