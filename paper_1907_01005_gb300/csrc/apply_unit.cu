// Register-resident matrix-free apply for p <= 2 (Alg. 6 restricted to the
// source pattern).
//
// One CTA processes one packed work unit: a patch and up to four of its
// column blocks (at most 32 columns, "lanes").  A thread owns one cell and
// LPT lanes (two for FP32, one for FP64): it holds all (p+1)^3 nodal values
// of its cell-columns in registers and applies the whole sum-factorised cell
// operator there -- interpolation to the Gauss points along x, y, z, the
// quadrature (three 1D Laplacian sweeps and the potential) and the
// transposed interpolation.  In FP32 the two columns go through packed
// FP32x2 FMAs, which halves the FMA instruction count.
//
// Data movement works on 16-byte row chunks (block rows are padded to 16
// bytes): the gather is a set of asynchronous 16-byte copies (cp.async, zero
// fill for absent blocks and boundary nodes) into a per-block patch tensor
// U_b[node][ld_b]; the cells add their results into a matching tensor with
// shared-memory atomics; the scatter adds 16-byte chunks into Y with vector
// reductions (red.global.add.v4.f32), 4x fewer than scalar atomics.
#include <algorithm>

#include "fe_internal.h"

namespace femf {
namespace {

// ---- lane arithmetic: packed FP32x2 FMA (sm_100+) or scalar FP64 -------
template <typename T, int LPT>
struct Lanes;
template <>
struct Lanes<float, 2> {       // two columns per thread, packed FP32x2 FMA
    using V = float2;
    static constexpr int n = 2;
    __device__ static V zero() { return make_float2(0.f, 0.f); }
    __device__ static V fma(float c, V a, V acc) { return __ffma2_rn(make_float2(c, c), a, acc); }
    __device__ static V make(float x0, float x1) { return make_float2(x0, x1); }
    __device__ static float get(V v, int i) { return i ? v.y : v.x; }
};
template <typename T>
struct Lanes<T, 1> {           // one column per thread
    using V = T;
    static constexpr int n = 1;
    __device__ static V zero() { return T(0); }
    __device__ static V fma(T c, V a, V acc) { return ::fma(c, a, acc); }
    __device__ static V make(T x0, T) { return x0; }
    __device__ static T get(V v, int) { return v; }
};

// 16-byte chunk of one block row added into Y
__device__ __forceinline__ void red_chunk(float* dst, const float* v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(dst), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]) : "memory");
}
__device__ __forceinline__ void red_chunk(double* dst, const double* v) {
    if (v[0] != 0.0) atomicAdd(dst, v[0]);
    if (v[1] != 0.0) atomicAdd(dst + 1, v[1]);
}

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

template <typename T, int P, int LPT_>
struct UnitGeo {
    static constexpr int N = P + 1, NP = 2 * P + 1, NPN = NP * NP * NP, N3 = N * N * N;
    static constexpr int L = kUnitLanes, LPT = LPT_, TPC = L / LPT;   // threads per cell
    static constexpr int THREADS = 8 * TPC;
    static constexpr int CH = 16 / sizeof(T);          // elements per 16-byte chunk
    static constexpr int MAXCH = kUnitLdSum / CH;      // chunks per node row of the unit
    // one work area: it holds the gathered patch tensor U_b[node][ld_b], and
    // after the cells have loaded their values into registers, the per-cell
    // output slices Yc_b[cell][local node][ld_b]
    static constexpr int TEN = (NPN > 8 * N3 ? NPN : 8 * N3) * kUnitLdSum;
    static constexpr size_t bytes = (size_t)(TEN + 8 * N3) * sizeof(T);
};

// resident CTAs per SM the register budget must allow: FP32 is bounded by
// shared memory at 5-6 CTAs of 8 warps, FP64 at 2-3 (the persistent loop
// otherwise lets the compiler keep loop-invariant values in registers and
// trade two resident CTAs for them)
template <typename T>
constexpr int kUnitMinBlocks = sizeof(T) == 4 ? 5 : 2;

template <typename T, int P, int LPT_>
__global__ void __launch_bounds__(UnitGeo<T, P, LPT_>::THREADS, kUnitMinBlocks<T>)
    apply_unit_kernel(const ApplyUnitArgs<T> a) {
    using G = UnitGeo<T, P, LPT_>;
    using LN = Lanes<T, LPT_>;
    using V = typename LN::V;
    constexpr int N = G::N, NP = G::NP, NPN = G::NPN, N3 = G::N3, L = G::L, LPT = G::LPT, TPC = G::TPC;
    constexpr int CH = G::CH, MAXCH = G::MAXCH;
    constexpr int SLOTS = MAXCH <= 16 ? 16 : 32;     // chunk slots per node (power of two)
    constexpr int SHIFT = SLOTS == 16 ? 4 : 5;
    static_assert(MAXCH <= SLOTS, "chunk slots");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* U = reinterpret_cast<T*>(smem_raw);         // per block b: [NPN][ld_b] at sBase[b]
    T* Yc = U;                                     // per block b: [8][N3][ld_b] at sBaseY[b] (after the loads)
    T* Vs = U + G::TEN;                            // [8][N3]  V at the Gauss points
    __shared__ int32_t sOff[kUnitBlocks][8];
    __shared__ int sLaneB[L], sLaneA[L], sMask[kUnitBlocks], sBase[kUnitBlocks], sBaseY[kUnitBlocks], sLd[kUnitBlocks], sW[kUnitBlocks];
    __shared__ unsigned short sList[NPN][8];       // (cell << 8) | local node, for the cells touching a node
    __shared__ unsigned char sCnt[NPN];
    __shared__ int sChB[SLOTS], sChC[SLOTS], sNch, sTen;
    __shared__ int sNode[NPN];                     // (slot << 16) | row, or -1 on the boundary

    __shared__ int64_t sItem;
    const int tid = threadIdx.x;
    constexpr int kElem16 = 16 / sizeof(T);      // elements per 16-byte offset unit
    // One unit per CTA, or (persistent launch) units pulled from a ticket
    // counter until the list is exhausted.
    int64_t item = blockIdx.x;
    if (a.ticket) {
        if (tid == 0) sItem = atomicAdd(a.ticket, 1ull);
        __syncthreads();
        item = sItem;
    }
    while (item < a.n_units) {
    const Unit& unit = a.units[item];
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
        sOff[tid >> 3][tid & 7] = (tid >> 3) < unit.nb ? unit.off[tid >> 3][tid & 7] : -1;
    }
    if (tid == 0) {
        int base = 0, basey = 0, nch = 0;
        for (int q = 0; q < kUnitBlocks; ++q) {
            const int ldq = q < unit.nb ? unit.ld[q] : 0;
            sBase[q] = base;
            sBaseY[q] = basey;
            sLd[q] = ldq;
            sW[q] = q < unit.nb ? unit.width[q] : 0;
            sMask[q] = q < unit.nb ? unit.cellmask[q] : 0;
            for (int c0 = 0; c0 < ldq; c0 += CH) { sChB[nch] = q; sChC[nch] = c0; ++nch; }
            base += NPN * ldq;
            basey += 8 * N3 * ldq;
        }
        sNch = nch;
        sTen = base;
    }
    for (int n = tid; n < NPN; n += blockDim.x) {
        sNode[n] = node_entry<P>(n, px, py, pz, a.lx, a.ly, a.lz, a.dirichlet);
        const int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
        int c = 0;
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx)
                    if (k >= cz * P && k <= cz * P + P && j >= cy * P && j <= cy * P + P && i >= cx * P && i <= cx * P + P)
                        sList[n][c++] = (unsigned short)(((cx + 2 * cy + 4 * cz) << 8) |
                                                         (((k - cz * P) * N + (j - cy * P)) * N + (i - cx * P)));
        sCnt[n] = (unsigned char)c;
    }
    __syncthreads();

    // ---- gather: asynchronous 16-byte copies of block row chunks ------------
    {
        const unsigned ubase = (unsigned)__cvta_generic_to_shared(U);
        const int nch = sNch;
        for (int e = tid; e < NPN * SLOTS; e += blockDim.x) {
            const int node = e >> SHIFT, j = e & (SLOTS - 1);
            if (j >= nch) continue;
            const int b = sChB[j], c0 = sChC[j], ld = sLd[b];
            const int ne = sNode[node];
            const int32_t o = ne >= 0 ? sOff[b][ne >> 16] : -1;
            const bool ok = o >= 0;
            const T* src = ok ? a.P + (int64_t)o * kElem16 + (ne & 0xffff) * ld + c0 : a.P;
            const unsigned dst = ubase + (unsigned)((sBase[b] + node * ld + c0) * sizeof(T));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                         "r"(ok ? 16 : 0) : "memory");
        }
        // the potential of the patch's cells (contiguous, 16-byte aligned)
        const T* Vg = a.Vq + (int64_t)unit.patch * 8 * N3;
        const unsigned vbase = (unsigned)__cvta_generic_to_shared(Vs);
        for (int e = tid; e < 8 * N3 / CH; e += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(vbase + 16u * e), "l"(Vg + e * CH) : "memory");
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();

    // ---- cell operator in registers -----------------------------------------
    {
        const int cell = tid / TPC, l0 = (tid % TPC) * LPT;
        const int cx = cell & 1, cy = (cell >> 1) & 1, cz = (cell >> 2) & 1;
        int lb[LPT], lofs[LPT], lld[LPT];
        bool act = false;
#pragma unroll
        for (int h = 0; h < LPT; ++h) {
            const int b = sLaneB[l0 + h];
            lb[h] = b;
            lld[h] = b >= 0 ? sLd[b] : 0;
            lofs[h] = b >= 0 ? sBase[b] + sLaneA[l0 + h] : 0;
            act |= b >= 0 && ((sMask[b] >> cell) & 1);
        }
        V u[N][N][N], t[N][N][N];
        if (act) {
#pragma unroll
            for (int z = 0; z < N; ++z)
#pragma unroll
                for (int y = 0; y < N; ++y)
#pragma unroll
                    for (int x = 0; x < N; ++x) {
                        const int node = ((cz * P + z) * NP + (cy * P + y)) * NP + (cx * P + x);
                        T v[LPT];
#pragma unroll
                        for (int h = 0; h < LPT; ++h) v[h] = lb[h] >= 0 ? U[lofs[h] + node * lld[h]] : T(0);
                        u[z][y][x] = LN::make(v[0], v[LPT - 1]);
                    }
        }
        __syncthreads();                                   // all inputs are in registers
        if (act) {
            const auto& K = a.k;
            // Sweeps run coefficient-outer: each (packed) coefficient is
            // loaded once and applied to all N^2 lines of the sweep.
#define SWEEP(C, IDX_D, IDX_S)                                               \
    _Pragma("unroll") for (int q = 0; q < N; ++q) {                          \
        _Pragma("unroll") for (int p2 = 0; p2 < N; ++p2) {                   \
            const T c = C[q][p2];                                            \
            _Pragma("unroll") for (int m = 0; m < N; ++m)                    \
            _Pragma("unroll") for (int n = 0; n < N; ++n) {                  \
                V& d = IDX_D;                                                \
                d = LN::fma(c, IDX_S, p2 == 0 ? LN::zero() : d);             \
            }                                                                \
        }                                                                    \
    }
            // interpolate to the Gauss points along x, y, z
            SWEEP(K.S, t[m][n][q], u[m][n][p2])
            SWEEP(K.S, u[m][q][n], t[m][p2][n])
            SWEEP(K.S, t[q][m][n], u[p2][m][n])
            // quadrature: V u_q plus the three collocation Laplacian sweeps
            // (|J| is folded into the coefficients: A / |J| here, |J| Sb in the
            // first transposed sweep below)
            const T* Vc = Vs + cell * N3;
#pragma unroll
            for (int z = 0; z < N; ++z)
#pragma unroll
                for (int y = 0; y < N; ++y)
#pragma unroll
                    for (int x = 0; x < N; ++x) u[z][y][x] = LN::fma(Vc[(z * N + y) * N + x], t[z][y][x], LN::zero());
#pragma unroll
            for (int q = 0; q < N; ++q)
#pragma unroll
                for (int l = 0; l < N; ++l) {
                    const T c0 = K.A[0][q][l], c1 = K.A[1][q][l], c2 = K.A[2][q][l];
#pragma unroll
                    for (int m = 0; m < N; ++m)
#pragma unroll
                        for (int n = 0; n < N; ++n) {
                            u[m][n][q] = LN::fma(c0, t[m][n][l], u[m][n][q]);
                            u[m][q][n] = LN::fma(c1, t[m][l][n], u[m][q][n]);
                            u[q][m][n] = LN::fma(c2, t[l][m][n], u[q][m][n]);
                        }
                }
            // integrate: transposed interpolation along x (with |J|), y, z
            SWEEP(K.Sb1, t[m][n][q], u[m][n][p2])
            SWEEP(K.Sb, u[m][q][n], t[m][p2][n])
            SWEEP(K.Sb, t[q][m][n], u[p2][m][n])
#undef SWEEP
            // the cell's output slice
#pragma unroll
            for (int h = 0; h < LPT; ++h) {
                if (lb[h] < 0) continue;
                T* dst = Yc + sBaseY[lb[h]] + (cell * N3) * lld[h] + sLaneA[l0 + h];
#pragma unroll
                for (int z = 0; z < N; ++z)
#pragma unroll
                    for (int y = 0; y < N; ++y)
#pragma unroll
                        for (int x = 0; x < N; ++x) dst[((z * N + y) * N + x) * lld[h]] = LN::get(t[z][y][x], h);
            }
        }
    }
    __syncthreads();

    // ---- scatter-add of 16-byte chunks (Alg. 6, write step) -----------------
    {
        const int nch = sNch;
        for (int e = tid; e < NPN * SLOTS; e += blockDim.x) {
            const int node = e >> SHIFT, j = e & (SLOTS - 1);
            if (j >= nch) continue;
            const int ne = sNode[node];
            if (ne < 0) continue;
            const int b = sChB[j], c0 = sChC[j], ld = sLd[b];
            const int32_t o = sOff[b][ne >> 16];
            if (o < 0) continue;
            // sum the slices of the (active) cells that touch the node; the
            // slices' padding columns hold stale data and are dropped
            T v[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q) v[q] = T(0);
            const int cnt = sCnt[node], mask = sMask[b];
            const T* yb = Yc + sBaseY[b] + c0;
            for (int c = 0; c < cnt; ++c) {
                const int ent = sList[node][c], cell = ent >> 8;
                if (!((mask >> cell) & 1)) continue;
                const T* src = yb + (cell * N3 + (ent & 0xff)) * ld;   // 16-byte aligned
                if constexpr (CH == 4) {
                    const float4 f = *reinterpret_cast<const float4*>(src);
                    v[0] += f.x; v[1] += f.y; v[2] += f.z; v[3] += f.w;
                } else {
#pragma unroll
                    for (int q = 0; q < CH; ++q) v[q] += src[q];
                }
            }
            const int w = sW[b];
            bool nz = false;
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                if (c0 + q >= w) v[q] = T(0);
                nz |= v[q] != T(0);
            }
            if (nz) red_chunk(a.Y + (int64_t)o * kElem16 + (ne & 0xffff) * ld + c0, v);
        }
    }
    }  // unit_ok
    if (!a.ticket) break;
    __syncthreads();                                   // shared tables are rebuilt for the next unit
    if (tid == 0) sItem = atomicAdd(a.ticket, 1ull);
    __syncthreads();
    item = sItem;
    }
}

template <typename T, int P, int LPT>
cudaError_t launch_units_p(const ApplyUnitArgs<T>& a, cudaStream_t s) {
    using G = UnitGeo<T, P, LPT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(apply_unit_kernel<T, P, LPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(apply_unit_kernel<T, P, LPT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (a.n_units == 0) return cudaSuccess;
    unsigned grid = (unsigned)a.n_units;
    if (a.ticket) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = (unsigned)std::min<int64_t>(a.n_units, (int64_t)sms * std::max(1, a.ctas_per_sm));
    }
    apply_unit_kernel<T, P, LPT><<<grid, G::THREADS, G::bytes, s>>>(a);
    return cudaGetLastError();
}

// columns per thread: FP32 runs one column per thread (more warps to hide the
// gather latency); FP64 one column per thread
template <typename T>
constexpr int kLanesPerThread = 1;

}  // namespace

template <typename T>
cudaError_t launch_apply_units(int p, const ApplyUnitArgs<T>& a, cudaStream_t s) {
    switch (p) {
        case 1: return launch_units_p<T, 1, kLanesPerThread<T>>(a, s);
        case 2: return launch_units_p<T, 2, kLanesPerThread<T>>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_apply_units<float>(int, const ApplyUnitArgs<float>&, cudaStream_t);
template cudaError_t launch_apply_units<double>(int, const ApplyUnitArgs<double>&, cudaStream_t);

}  // namespace femf
