// Device helpers shared by the apply kernels (apply_unit.cu: sum
// factorisation in registers; apply_cellmat.cu: cell matrices on the tensor
// cores; apply.cu: the p >= 3 plane kernel): the patch-node table, the
// fixed-order sum of the cells' results, and the conflict-free write of a
// patch's results into Y.
//
// Write into Y (Alg. 6, write step, with the "compress" of Sec. 3.4 done on
// the device).  Row block r is owned by its patch; its upper-face nodes also
// receive contributions from the upper neighbour patches r + e, e in
// {0,1}^3 \ {0}.  Work items are taken in descending patch rank (Morton
// ranks grow with each coordinate, so upper neighbours come first).  Each
// work item (1) stores its contributions to its lower neighbours' rows in
// halo slots of their own (block, e), then marks its patch; (2) waits,
// bounded in time, until its (at most 7) upper neighbours have marked theirs;
// (3) fetches the halo rows addressed to its own blocks into shared memory
// (one round of asynchronous copies), adds them to its own rows in a fixed
// order (own part, then e = 1 .. 7), and stores every row of its own blocks
// once.
// No step waits on anything but halo writes, which never wait, so the waits
// stay one level deep.  Y gets no zero-fill, no atomics and no
// read-modify-write, and the same bits on every run.
#pragma once

#include "fe_internal.h"

namespace femf {
namespace {

// Node `node` of the (2p+1)^3 patch (px, py, pz): row (bits 0-15) of the
// node in the row block that owns it, that row block's slot s = dx + 2 dy +
// 4 dz (bits 16-18; the owner is patch (px - 1 + dx, py - 1 + dy, pz - 1 +
// dz), s = 7 the patch itself), kBoundary for a Dirichlet boundary node
// (input read as zero, output zero), and in bits 22-30: for an own node its
// face mask f (f_d = 1 on the upper face in direction d when an upper
// neighbour exists there), else its index in the owner's halo slot.
constexpr int kBoundary = 1 << 21;
constexpr int kAuxShift = 22;

// Index of an owner-frame node (i, j, k) of patch (px, py, pz) in the halo
// slot of offset e: lexicographic (x fastest) over the directions d with
// e_d = 0, each over the owner's node range [lo, 2p], lo = 0 for a patch at
// coordinate 0 and 1 else.
template <int P>
__device__ __forceinline__ int halo_face_index(int e, int i, int j, int k, int px, int py, int pz) {
    constexpr int Q = 2 * P;
    int idx = 0, stride = 1;
    if (!(e & 1)) { const int lo = px > 0; idx += (i - lo) * stride; stride *= Q + 1 - lo; }
    if (!(e & 2)) { const int lo = py > 0; idx += (j - lo) * stride; stride *= Q + 1 - lo; }
    if (!(e & 4)) { const int lo = pz > 0; idx += (k - lo) * stride; }
    return idx;
}

template <int P>
__device__ __forceinline__ int node_entry(int node, int px, int py, int pz, int lx, int ly, int lz, int dirichlet,
                                          int npx, int npy, int npz) {
    constexpr int Q = 2 * P, NP = 2 * P + 1;
    const int i = node % NP, j = (node / NP) % NP, k = node / (NP * NP);
    const int I = Q * px + i, J = Q * py + j, K = Q * pz + k;
    const int dx = (i == 0 && px > 0) ? 0 : 1;
    const int dy = (j == 0 && py > 0) ? 0 : 1;
    const int dz = (k == 0 && pz > 0) ? 0 : 1;
    const int ii = dx ? i : Q, jj = dy ? j : Q, kk = dz ? k : Q;
    const int qx = px - 1 + dx, qy = py - 1 + dy, qz = pz - 1 + dz;
    const int nxq = Q + (qx == 0), nyq = Q + (qy == 0);
    const int row = (ii - (qx != 0)) + nxq * ((jj - (qy != 0)) + nyq * (kk - (qz != 0)));
    const int slot = dx + 2 * dy + 4 * dz;
    int aux;
    if (slot == 7)
        aux = (i == Q && px + 1 < npx ? 1 : 0) | (j == Q && py + 1 < npy ? 2 : 0) | (k == Q && pz + 1 < npz ? 4 : 0);
    else
        aux = halo_face_index<P>(7 - slot, i, j, k, px, py, pz);   // free directions: the owner's coordinates are ours
    const bool bnd = dirichlet && (I == 0 || J == 0 || K == 0 || I == lx - 1 || J == ly - 1 || K == lz - 1);
    return (slot << 16) | row | (bnd ? kBoundary : 0) | (aux << kAuxShift);
}

constexpr uint64_t kOrderWaitNs = 500ull * 1000 * 1000;   // bounded wait for neighbour patches (0.5 s)

__device__ __forceinline__ uint64_t order_clock_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Called by all threads of warp 0: lane e in 1..7 waits until the upper
// neighbour (px, py, pz) + e, if it exists, has written its halo
// (done[pid] == count[pid], both indexed by pid = x + npx (y + npy z)).
// Returns false (in every lane) when a wait gave up.
__device__ __forceinline__ bool wait_upper_neighbours(const int32_t* done, const int32_t* count, int px, int py,
                                                      int pz, int npx, int npy, int npz) {
    const int e = threadIdx.x & 31;
    bool ok = true;
    if (e >= 1 && e < 8) {
        const int qx = px + (e & 1), qy = py + ((e >> 1) & 1), qz = pz + (e >> 2);
        if (qx < npx && qy < npy && qz < npz) {
            const int q = qx + npx * (qy + npy * qz);
            const int want = count[q];
            const uint64_t t0 = order_clock_ns();
            while (true) {
                int v;
                asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(done + q) : "memory");
                if (v >= want) break;
                if (order_clock_ns() - t0 > kOrderWaitNs) {
                    ok = false;
                    break;
                }
            }
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// Called by thread 0 after a __syncthreads that follows the CTA's halo
// stores: publishes one work item of patch pid whose halo is written.
__device__ __forceinline__ void mark_done(int32_t* done, int pid) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(done + pid), "r"(1) : "memory");
}

// 16-byte vectors of the rows (ld, the row stride, is a multiple of 16 bytes)
template <typename T> struct V16;
template <> struct V16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static void add(float4& a, const float4& b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }
};
template <> struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static void add(double2& a, const double2& b) { a.x += b.x; a.y += b.y; }
};

// A row of the patch tensor (ys) to a halo row (dst).  Stores go to L2 only:
// another SM reads them.
template <typename T>
__device__ __forceinline__ void put_halo_row(T* dst, const T* ys, int ld) {
    using V = typename V16<T>::type;
    for (int c0 = 0; c0 < ld; c0 += V16<T>::n)
        __stcg(reinterpret_cast<V*>(dst + c0), *reinterpret_cast<const V*>(ys + c0));
}

// Rows of the halo slot of upper-neighbour offset e for an own block of
// patch (px, py, pz): the product over the directions with e_d = 0 of the
// own node range 2p + [p_d == 0].
template <int P>
__device__ __forceinline__ int halo_slot_rows(int e, int px, int py, int pz) {
    constexpr int Q = 2 * P;
    return ((e & 1) ? 1 : Q + (px == 0)) * ((e & 2) ? 1 : Q + (py == 0)) * ((e & 4) ? 1 : Q + (pz == 0));
}

// Copies the halo slots addressed to a work item's own blocks into shared
// memory with 16-byte asynchronous copies, so that the own rows are summed
// from shared memory: slot (b, e) of nslot[b][e] elements (0 where there is
// none; a whole number of 16-byte chunks) from halo + hin[b][e] 16-byte units
// to hbuf + base[b][e], the slots packed in the order (b, e).  base is filled
// here by warp 0 (a prefix sum over the at most 32 slots).  The chunks of all
// slots are then dealt to the threads in one flat range: a thread first
// works out the source and destination of each of its chunks (a binary search
// over the slot starts) and only then issues its copies back to back.  The
// caller waits (cp.async.wait_all) and synchronises before reading hbuf.
template <typename T>
__device__ __forceinline__ void fetch_halo(T* hbuf, const T* halo, const int32_t (*hin)[8], const int (*nslot)[8],
                                           int (*base)[8], int nblocks) {
    constexpr int CH = 16 / sizeof(T);
    if (threadIdx.x < 32) {
        const int b = threadIdx.x >> 3, e = threadIdx.x & 7;
        const int n = b < nblocks ? nslot[b][e] : 0;
        int v = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if ((int)(threadIdx.x & 31) >= o) v += y;
        }
        if (b < nblocks) base[b][e] = v - n;
    }
    __syncthreads();
    if (nblocks <= 0) return;
    const int nq = 8 * nblocks;                       // slots q = 8 b + e
    const int* bflat = &base[0][0];
    const int total = (bflat[nq - 1] + nslot[nblocks - 1][7]) / CH;
    const unsigned dst0 = (unsigned)__cvta_generic_to_shared(hbuf);
    constexpr int K = 4;                              // chunks per thread resolved before issuing
    for (int c0 = 0; c0 < total; c0 += K * (int)blockDim.x) {
        const T* src[K];
        unsigned dst[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int c = c0 + (int)threadIdx.x + k * (int)blockDim.x;
            src[k] = nullptr;
            dst[k] = 0u;
            if (c < total) {
                // the last slot q with base <= c * CH (empty slots share their
                // start with the next one, so q is the slot holding chunk c)
                int q = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (q + step < nq && bflat[q + step] <= c * CH) q += step;
                const int r = c * CH - bflat[q];
                src[k] = halo + (int64_t)hin[q >> 3][q & 7] * CH + r;
                dst[k] = dst0 + (unsigned)((bflat[q] + r) * (int)sizeof(T));
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (src[k] != nullptr)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst[k]), "l"(src[k]) : "memory");
    }
}

// Own row r of patch (px, py, pz), rows x fastest over the own range [l, 2p]
// per direction (l = 0 at coordinate 0, else 1): the node and its own-range
// coordinates packed as node | rx << 10 | ry << 14 | rz << 18 (built once per
// work item by own_row_entry, read by store_own_rows).
template <int P>
__device__ __forceinline__ int own_row_entry(int r, int px, int py, int pz) {
    constexpr int Q = 2 * P, NP = 2 * P + 1;
    const int lx = px > 0, ly = py > 0, lz = pz > 0;
    // the own range has 2p or 2p + 1 nodes: divisions by constants
    const int rx = lx ? r % Q : r % (Q + 1), ryz = lx ? r / Q : r / (Q + 1);
    const int ry = ly ? ryz % Q : ryz % (Q + 1), rz = ly ? ryz / Q : ryz / (Q + 1);
    const int node = (lx + rx) + NP * ((ly + ry) + NP * (lz + rz));
    return node | (rx << 10) | (ry << 14) | (rz << 18);
}
template <int P>
__device__ __forceinline__ int own_rows_of(int px, int py, int pz) {
    constexpr int Q = 2 * P;
    return (Q + 1 - (px > 0)) * (Q + 1 - (py > 0)) * (Q + 1 - (pz > 0));
}

// Stores the own rows of every block into Y: the patch's part (the patch
// tensor yp: node row stride S elements, block b at column colbase[b], ld[b]
// columns) plus the fetched halo rows of the upper neighbours e within the
// node's face mask (slot (b, e) at hbuf + hb[b][e] where nslot[b][e] > 0,
// the row at its halo_face_index), added in the order e = 1 .. 7, so every
// row has the same rounding on every run; zeros for boundary nodes.  Block
// b's own rows form one contiguous range of Y starting at own_row0(b) (rows
// x fastest over the own range; own_tab[r] = own_row_entry(r), or nullptr
// to decode each row where it is used), so the
// threads take its 16-byte chunks in address order and a warp's stores
// cover consecutive addresses.  Blocks with no own rows here have
// own_row0(b) == nullptr.
template <int P, typename T, typename OwnRow0>
__device__ __forceinline__ void store_own_rows(OwnRow0 own_row0, const T* yp, int S, const int* colbase,
                                               const int* ld, const T* hbuf, const int (*hb)[8],
                                               const int (*nslot)[8], const int* node_tab, const int* own_tab,
                                               int nblocks, int px, int py, int pz) {
    using V = typename V16<T>::type;
    constexpr int CH = 16 / sizeof(T), Q = 2 * P;
    const int nx = Q + 1 - (px > 0), ny = Q + 1 - (py > 0);
    const int rows = own_rows_of<P>(px, py, pz);
    for (int b = 0; b < nblocks; ++b) {
        T* yd = own_row0(b);
        if (yd == nullptr) continue;
        const int ldb = ld[b], cpr = ldb / CH, total = rows * cpr;
        const float inv_cpr = 1.0f / (float)cpr;      // c / cpr exactly for these small c
        int hbe[8];                                    // slot starts, -1 where there is no halo
#pragma unroll
        for (int e = 1; e < 8; ++e) hbe[e] = nslot[b][e] > 0 ? hb[b][e] : -1;
        for (int c = threadIdx.x; c < total; c += blockDim.x) {
            const int r = __float2int_rz(((float)c + 0.5f) * inv_cpr), cc = c - r * cpr;
            const int ow = own_tab != nullptr ? own_tab[r] : own_row_entry<P>(r, px, py, pz);
            const int node = ow & 1023, rx = (ow >> 10) & 15, ry = (ow >> 14) & 15, rz = (ow >> 18) & 15;
            const int ne = node_tab[node];
            V v = V16<T>::zero();
            if (!(ne & kBoundary)) {
                v = *reinterpret_cast<const V*>(yp + node * S + colbase[b] + cc * CH);
                const int f = (ne >> kAuxShift) & 7;
                if (f) {
#pragma unroll
                    for (int e = 1; e < 8; ++e) {
                        if ((f & e) != e || hbe[e] < 0) continue;
                        // halo_face_index in own-range coordinates: the free
                        // directions (e_d = 0), x fastest
                        int idx = 0, st = 1;
                        if (!(e & 1)) { idx += rx * st; st *= nx; }
                        if (!(e & 2)) { idx += ry * st; st *= ny; }
                        if (!(e & 4)) idx += rz * st;
                        V16<T>::add(v, *reinterpret_cast<const V*>(hbuf + hbe[e] + idx * ldb + cc * CH));
                    }
                }
            }
            __stcg(reinterpret_cast<V*>(yd) + c, v);
        }
    }
}

// Sums the results of the eight cells of a patch in a fixed order and stores
// every patch node once, for CTAs of 256 threads where thread (cell =
// tid / 32, lane = tid % 32) holds t, its cell's (p+1)^3 results for one
// column lane.  Cells that share nodes are merged pairwise: along x (cell
// cx = 1 hands its x = 0 face to cell cx = 0, which adds it into its x = p
// face), then along y, then along z, through the exchange buffer ex (free
// shared memory of 2 kMergeFace<P> elements: the faces alternate between two
// halves; with SINGLE one half and a barrier more per step).  Afterwards a cell owns its local nodes with x >= cx,
// y >= cy, z >= cz, and each patch node has exactly one owner, which stores
// it (plain store) at yp[base + ((z NP + y) NP + x) S].  With the faces merged
// in this order every node's sum has the same rounding on every run.  Every
// thread of the CTA must call it (it holds barriers); `store` is false for
// lanes without a column.
template <int P>
constexpr int kMergeFace = (P + 1) * (P + 1) * 256;   // one face of every thread
template <int P, int S, int NP, bool SINGLE, typename T>
__device__ __forceinline__ void merge_cells_store(T (&t)[P + 1][P + 1][P + 1], int cell, int lane, bool store, T* ex,
                                                  T* yp, int base) {
    constexpr int N = P + 1;
    const int cx = cell & 1, cy = (cell >> 1) & 1, cz = (cell >> 2) & 1;
    // slot of face entry f of the receiving cell rc: [f][rc][lane]
    auto slot = [&](T* e, int f, int rc) -> T& { return e[(f * 8 + rc) * 32 + lane]; };
    T* e0 = ex;
    T* e1 = SINGLE ? ex : ex + kMergeFace<P>;
    // x: cell cx = 1 sends its x = 0 face to cell cell - 1
    if (cx) {
#pragma unroll
        for (int z = 0; z < N; ++z)
#pragma unroll
            for (int y = 0; y < N; ++y) slot(e0, z * N + y, cell - 1) = t[z][y][0];
    }
    __syncthreads();
    if (!cx) {
#pragma unroll
        for (int z = 0; z < N; ++z)
#pragma unroll
            for (int y = 0; y < N; ++y) t[z][y][P] += slot(e0, z * N + y, cell);
    }
    if (SINGLE) __syncthreads();
    // y: cell cy = 1 sends its y = 0 face to cell cell - 2
    if (cy) {
#pragma unroll
        for (int z = 0; z < N; ++z)
#pragma unroll
            for (int x = 0; x < N; ++x) slot(e1, z * N + x, cell - 2) = t[z][0][x];
    }
    __syncthreads();
    if (!cy) {
#pragma unroll
        for (int z = 0; z < N; ++z)
#pragma unroll
            for (int x = 0; x < N; ++x) t[z][P][x] += slot(e1, z * N + x, cell);
    }
    if (SINGLE) __syncthreads();
    // z: cell cz = 1 sends its z = 0 face to cell cell - 4
    if (cz) {
#pragma unroll
        for (int y = 0; y < N; ++y)
#pragma unroll
            for (int x = 0; x < N; ++x) slot(e0, y * N + x, cell - 4) = t[0][y][x];
    }
    __syncthreads();
    if (!cz) {
#pragma unroll
        for (int y = 0; y < N; ++y)
#pragma unroll
            for (int x = 0; x < N; ++x) t[P][y][x] += slot(e0, y * N + x, cell);
    }
    if (store) {
#pragma unroll
        for (int z = 0; z < N; ++z)
#pragma unroll
            for (int y = 0; y < N; ++y)
#pragma unroll
                for (int x = 0; x < N; ++x)
                    if (x >= cx && y >= cy && z >= cz) yp[base + ((z * NP + y) * NP + x) * S] = t[z][y][x];
    }
}

}  // namespace
}  // namespace femf
