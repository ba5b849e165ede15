// Matrix-free application of H = -1/2 Laplacian + V to a BCSR multivector
// (Alg. 6 with the destination restricted to the source pattern).
//
// One CTA processes one (patch, column block) tile: it gathers the patch's
// (2p+1)^3 nodal values of the column block from up to eight stored blocks
// (the patch's own row block and its seven lower neighbours, Alg. 4/5
// semantics precomputed into the tile), runs the sum-factorised cell operator
// on each of the patch's eight cells, accumulates the cell results into a
// patch tensor in shared memory and writes the patch tensor into Y in the
// conflict-free write of unit_common.cuh (tiles taken in descending patch
// rank from a work counter; contributions to lower neighbours through halo
// slots; every own row stored once; no zero-fill of Y, no global atomics).
//
// Thread mapping: a thread owns one (cell, column, plane) triple.  A cell
// column is an n^3 tensor (n = p+1); its n threads each hold an n x n plane in
// registers, so the 1D contractions along the two in-plane directions are
// register-only and the third direction is reached by an exchange through
// shared memory (z-planes <-> y-planes).
#include <cstdio>

#include "fe_internal.h"
#include "unit_common.cuh"

namespace femf {
namespace {

template <int P>
struct Geo {
    static constexpr int N = P + 1;          // nodes / Gauss points per cell direction
    static constexpr int NP = 2 * P + 1;     // patch nodes per direction
    static constexpr int NPN = NP * NP * NP;
    static constexpr int N3 = N * N * N;
};

// Threads per CTA are capped so that the per-thread planes (four n x n arrays)
// stay in registers: 8 cells x 16 columns x n planes for p <= 2, half of that
// for p >= 3.
template <int P>
constexpr int max_threads() { return (P >= 3 ? 4 : 8) * kMaxW * (P + 1); }

template <typename T, int P, bool MASS>
__global__ void __launch_bounds__(max_threads<P>()) apply_plane_kernel(const ApplyArgs<T> a) {
    using G = Geo<P>;
    constexpr int N = G::N, NP = G::NP, NPN = G::NPN, N3 = G::N3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wmax = a.wmax;
    const int cpr = a.cells_per_round;
    const int ldmax = a.ldmax;
    T* U = reinterpret_cast<T*>(smem_raw);          // [NPN][ld] gathered input (capacity NPN * ldmax)
    T* Yp = U + NPN * ldmax;                         // [NPN][ld] accumulated output (16-byte aligned)
    T* exA = Yp + NPN * ldmax;                       // [cpr*wmax][N3] exchange
    T* exB = exA + cpr * wmax * N3;

    // tiles in descending order (descending patch rank, the order of the write)
    __shared__ int64_t sTicket;
    if (threadIdx.x == 0) sTicket = (int64_t)atomicAdd(a.ticket, 1ull);
    __syncthreads();
    if (sTicket >= a.n_tiles) return;
    const Tile& tile = a.tiles[a.n_tiles - 1 - sTicket];
    const int w = tile.width, ld = tile.ld;
    const int px = tile.pxyz & 1023, py = (tile.pxyz >> 10) & 1023, pz = tile.pxyz >> 20;
    const int cellmask = tile.cellmask;
    const bool in_mesh = px < a.npx && py < a.npy && pz < a.npz;
    if (!in_mesh || w > wmax || w < 1 || ld < w || ld > ldmax || ld % (16 / (int)sizeof(T)) != 0 ||
        ldmax % (16 / (int)sizeof(T)) != 0) {
        // a malformed tile: reported, skipped, and counted as finished so
        // that its neighbours do not wait for it
        if (threadIdx.x == 0) {
            atomicExch(a.status, kDevBadTile);
            if (in_mesh) mark_done(a.done, px + a.npx * (py + a.npy * pz));
        }
        return;
    }
    __shared__ int64_t sOff[8];
    __shared__ int32_t sHout[8], sHin[1][8];
    __shared__ int sHn[1][8], sHb[1][8];              // fetched halo slots: elements, buffer offsets
    __shared__ int sCol0[1], sLd1[1];                 // the tile's one block: column 0, ld columns
    __shared__ int sNode[NPN];                       // node_entry: row, owner slot, boundary bit, face data
    if (threadIdx.x < 8) {
        sOff[threadIdx.x] = tile.off[threadIdx.x];
        sHout[threadIdx.x] = tile.hout[threadIdx.x];
        sHin[0][threadIdx.x] = tile.hin[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        sCol0[0] = 0;
        sLd1[0] = ld;
    }
    for (int n = threadIdx.x; n < NPN; n += blockDim.x)
        sNode[n] = node_entry<P>(n, px, py, pz, a.lx, a.ly, a.lz, a.dirichlet, a.npx, a.npy, a.npz);
    __syncthreads();
    constexpr int CH = 16 / sizeof(T);               // elements per 16-byte chunk (ld is a multiple)

    // ---- gather (Alg. 6, read step): 16-byte asynchronous copies, one task
    // per node row (the node table is read once, then the row's chunks) ------
    {
        const unsigned ubase = (unsigned)__cvta_generic_to_shared(U);
        for (int node = threadIdx.x; node < NPN; node += blockDim.x) {
            const int ne = sNode[node];
            const int64_t o = (ne & kBoundary) ? -1 : sOff[(ne >> 16) & 7];
            const bool ok = o >= 0;
            const T* src = ok ? a.P + o + (int64_t)(ne & 0xffff) * ld : a.P;
            const unsigned dst = ubase + (unsigned)(node * ld * sizeof(T));
            for (int c0 = 0; c0 < ld; c0 += CH)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + c0 * (int)sizeof(T)),
                             "l"(ok ? src + c0 : src), "r"(ok ? 16 : 0) : "memory");
        }
        for (int e = threadIdx.x; e < NPN * ld / CH; e += blockDim.x)
            reinterpret_cast<uint4*>(Yp)[e] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();

    // ---- cell operator, cpr cells at a time ------------------------------
    const int t = threadIdx.x % N;            // plane index
    const int cc = threadIdx.x / N;           // cell-column slot in this round
    const int col = cc % wmax;
    const int cslot = cc / wmax;
    const auto& K = a.k;
    T* myA = exA + (size_t)cc * N3;
    T* myB = exB + (size_t)cc * N3;

    for (int c0 = 0; c0 < 8; c0 += cpr) {
        const int cell = c0 + cslot;
        const bool act = (cslot < cpr) && (col < w) && ((cellmask >> cell) & 1);
        const int cx = cell & 1, cy = (cell >> 1) & 1, cz = (cell >> 2) & 1;
        T pa[N][N], pb[N][N];
        // z-plane t of nodal values: pa[j][i]
        if (act) {
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int node = (cx * P + i) + NP * ((cy * P + j) + NP * (cz * P + t));
                    pa[j][i] = U[node * ld + col];
                }
            // interpolate along x then y: pa -> pb -> pa  (values at (q_x, q_y, node z=t))
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    T s = T(0);
#pragma unroll
                    for (int i = 0; i < N; ++i) s = fma(K.S[q][i], pa[j][i], s);
                    pb[j][q] = s;
                }
#pragma unroll
            for (int q = 0; q < N; ++q)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T s = T(0);
#pragma unroll
                    for (int j = 0; j < N; ++j) s = fma(K.S[q][j], pb[j][i], s);
                    pa[q][i] = s;
                }
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) myA[(t * N + j) * N + i] = pa[j][i];
        }
        __syncthreads();
        // y-own: thread t holds q_y = t; pa[k][i] = value at (q_x=i, q_y=t, node z=k)
        T uq[N][N], z1[N][N];
        if (act) {
#pragma unroll
            for (int k = 0; k < N; ++k)
#pragma unroll
                for (int i = 0; i < N; ++i) pa[k][i] = myA[(k * N + t) * N + i];
            // interpolate along z
#pragma unroll
            for (int q = 0; q < N; ++q)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T s = T(0);
#pragma unroll
                    for (int k = 0; k < N; ++k) s = fma(K.S[q][k], pa[k][i], s);
                    uq[q][i] = s;
                }
            // quadrature: x and z Laplacian terms and the potential (the mass
            // operator: |J| u_q only)
            const T* V = MASS ? nullptr : a.Vq + ((int64_t)tile.patch * 8 + cell) * N3;
#pragma unroll
            for (int kq = 0; kq < N; ++kq)
#pragma unroll
                for (int iq = 0; iq < N; ++iq) {
                    T s = MASS ? K.jxw * uq[kq][iq] : K.jxw * V[iq + N * (t + N * kq)] * uq[kq][iq];
                    if constexpr (!MASS) {
#pragma unroll
                        for (int l = 0; l < N; ++l) s = fma(K.A[0][iq][l], uq[kq][l], s);
#pragma unroll
                        for (int l = 0; l < N; ++l) s = fma(K.A[2][kq][l], uq[l][iq], s);
                    }
                    z1[kq][iq] = s;
                }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k = 0; k < N; ++k)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    myA[(k * N + t) * N + i] = uq[k][i];
                    myB[(k * N + t) * N + i] = z1[k][i];
                }
        }
        __syncthreads();
        if (act) {
            // z-own: thread t holds q_z = t; add the y Laplacian term
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    pa[j][i] = myA[(t * N + j) * N + i];   // u_q
                    pb[j][i] = myB[(t * N + j) * N + i];   // partial sum
                }
#pragma unroll
            for (int jq = 0; jq < N; ++jq)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T s = pb[jq][i];
                    if constexpr (!MASS) {
#pragma unroll
                        for (int l = 0; l < N; ++l) s = fma(K.A[1][jq][l], pa[l][i], s);
                    }
                    z1[jq][i] = s;
                }
            // integrate along x then y: z1 -> pb -> pa  (nodal x, nodal y, q_z = t)
#pragma unroll
            for (int jq = 0; jq < N; ++jq)
#pragma unroll
                for (int ia = 0; ia < N; ++ia) {
                    T s = T(0);
#pragma unroll
                    for (int iq = 0; iq < N; ++iq) s = fma(K.Sb[ia][iq], z1[jq][iq], s);
                    pb[jq][ia] = s;
                }
#pragma unroll
            for (int ja = 0; ja < N; ++ja)
#pragma unroll
                for (int ia = 0; ia < N; ++ia) {
                    T s = T(0);
#pragma unroll
                    for (int jq = 0; jq < N; ++jq) s = fma(K.Sb[ja][jq], pb[jq][ia], s);
                    pa[ja][ia] = s;
                }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) myA[(t * N + j) * N + i] = pa[j][i];
        }
        __syncthreads();
        if (act) {
            // y-own: thread t holds nodal y = t; integrate along z and accumulate
#pragma unroll
            for (int k = 0; k < N; ++k)
#pragma unroll
                for (int i = 0; i < N; ++i) pb[k][i] = myA[(k * N + t) * N + i];
#pragma unroll
            for (int ka = 0; ka < N; ++ka)
#pragma unroll
                for (int ia = 0; ia < N; ++ia) {
                    T s = T(0);
#pragma unroll
                    for (int kq = 0; kq < N; ++kq) s = fma(K.Sb[ka][kq], pb[kq][ia], s);
                    pa[ka][ia] = s;
                }
        }
        // add the cells' results into the patch tensor one cell slot at a
        // time (cells share face, edge and centre nodes): a fixed order of
        // the additions, and no two threads of a phase touch the same node
        for (int k = 0; k < cpr; ++k) {
            if (act && cslot == k) {
#pragma unroll
                for (int ka = 0; ka < N; ++ka)
#pragma unroll
                    for (int ia = 0; ia < N; ++ia) {
                        const int node = (cx * P + ia) + NP * ((cy * P + t) + NP * (cz * P + ka));
                        Yp[node * ld + col] += pa[ka][ia];
                    }
            }
            __syncthreads();
        }
    }

    // ---- write into Y (Alg. 6, write step; unit_common.cuh), one task per
    // node row: (1) contributions to the lower neighbours' rows into their
    // halo slots, (2) wait for the upper neighbours' halos, (3) own rows --------
    constexpr int kElem16 = 16 / sizeof(T);
    for (int node = threadIdx.x; node < NPN; node += blockDim.x) {
        const int ne = sNode[node];
        const int slot = (ne >> 16) & 7;
        if (slot == 7 || (ne & kBoundary)) continue;
        const int32_t h = sHout[slot];
        if (h < 0) continue;
        put_halo_row(a.halo + (int64_t)h * kElem16 + (ne >> kAuxShift) * ld, Yp + node * ld, ld);
    }
    __syncthreads();
    // the patch is marked by a thread outside warp 0 while warp 0 waits for
    // the neighbours
    if (threadIdx.x == (blockDim.x > 32 ? 32u : 0u)) mark_done(a.done, px + a.npx * (py + a.npy * pz));
    if (threadIdx.x < 32 && !wait_upper_neighbours(a.done, a.count, px, py, pz, a.npx, a.npy, a.npz) &&
        threadIdx.x == 0)
        atomicExch(a.status, kDevTimeout);
    const int64_t oown = sOff[7];
    // the halos addressed to this tile, fetched into the free gather buffer
    // (slot sizes by lanes 0..7 of warp 0, the lanes that read them in the
    // prefix of fetch_halo; its barrier publishes them)
    if (threadIdx.x < 8) {
        const int e = threadIdx.x;
        sHn[0][e] = (e > 0 && oown >= 0 && sHin[0][e] >= 0) ? halo_slot_rows<P>(e, px, py, pz) * ld : 0;
    }
    fetch_halo(U, a.halo, sHin, sHn, sHb, 1);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // own rows: own part plus the halo rows, stored once
    store_own_rows<P>([&](int) -> T* { return oown >= 0 ? a.Y + oown : nullptr; }, Yp, ld, sCol0, sLd1, U, sHb, sHn,
                      sNode, nullptr, 1, px, py, pz);
}

template <typename T, int P>
cudaError_t launch_p(const ApplyArgs<T>& a, cudaStream_t s) {
    const size_t smem = apply_smem_bytes<T>(P, a.wmax, a.ldmax, a.cells_per_round);
    const int threads = apply_threads<T>(P, a.wmax, a.cells_per_round);
    // dynamic shared memory up to 223 KB: the node and halo tables take about 3 KB of the 227 KB a CTA may use
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(apply_plane_kernel<T, P, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 223 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(apply_plane_kernel<T, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     223 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.n_tiles == 0) return cudaSuccess;
    if (a.mass)
        apply_plane_kernel<T, P, true><<<(unsigned)a.n_tiles, threads, smem, s>>>(a);
    else
        apply_plane_kernel<T, P, false><<<(unsigned)a.n_tiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
size_t apply_smem_bytes(int p, int wmax, int ldmax, int cpr) {
    const size_t np = 2 * p + 1, n = p + 1;
    return (2 * np * np * np * ldmax + 2 * (size_t)cpr * wmax * n * n * n) * sizeof(T);
}

int apply_max_threads(int p) {
    switch (p) {
        case 1: return max_threads<1>();
        case 2: return max_threads<2>();
        case 3: return max_threads<3>();
        default: return max_threads<4>();
    }
}

template <typename T>
int apply_threads(int p, int wmax, int cpr) {
    const int t = cpr * wmax * (p + 1);
    return (t + 31) / 32 * 32;
}

template <typename T>
cudaError_t launch_apply(int p, const ApplyArgs<T>& a, cudaStream_t s) {
    switch (p) {
        case 1: return launch_p<T, 1>(a, s);
        case 2: return launch_p<T, 2>(a, s);
        case 3: return launch_p<T, 3>(a, s);
        case 4: return launch_p<T, 4>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_apply<float>(int, const ApplyArgs<float>&, cudaStream_t);
template cudaError_t launch_apply<double>(int, const ApplyArgs<double>&, cudaStream_t);
template size_t apply_smem_bytes<float>(int, int, int, int);
template size_t apply_smem_bytes<double>(int, int, int, int);
template int apply_threads<float>(int, int, int);
template int apply_threads<double>(int, int, int);

}  // namespace femf
