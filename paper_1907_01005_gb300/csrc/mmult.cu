// Post-multiplication of a BCSR multivector by a small dense matrix, with a
// destination pattern (Alg. 7, Sec. 3.6; Eqs. G_ops1/G_ops2), and the
// column-wise inner product tr(D^T G) (Eq. G_ops4).
//
// C = alpha (A X + gamma A) + beta C, where A and C share one block pattern
// and X is M x M.  Row block r of the product only needs the columns of r's
// own stored blocks (its "union"): C_r = A_r X[union, union], a dense
// (rows_r x W_r) by (W_r x W_r) product; the products A_rk X_kj whose column
// block j is not stored in row block r are the ones Alg. 7 discards.
//
// Work item: (row block, 64-row chunk, 64-column chunk of the union).  256
// threads, each owning a 4 x 4 micro-tile; the union is walked in k-tiles of
// 32 columns staged in shared memory (X rounded to the working precision).
#include <algorithm>
#include <type_traits>

#include "fe_internal.h"

namespace femf {
namespace {

constexpr int kMT = 64;          // rows per tile
constexpr int kNT = 64;          // output columns per tile
constexpr int kKT = 32;          // union columns per k-step

template <typename T>
__global__ void __launch_bounds__(256) mmult_kernel(const MmultArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int64_t* sUoff = reinterpret_cast<int64_t*>(smem_raw);     // [wmax] element offset of column u in row 0
    int* sUld = reinterpret_cast<int*>(sUoff + a.wmax_union);   // [wmax] row stride
    int* sUcol = sUld + a.wmax_union;                           // [wmax] global column
    __shared__ T sA[kMT][kKT + 1];
    __shared__ T sX[kKT][kNT + 1];

    const MmultItem it = a.items[blockIdx.x];
    const int tid = threadIdx.x;
    const int r = it.r;
    const int64_t b0 = a.row_ptr[r], b1 = a.row_ptr[r + 1];
    const int W = a.rb_union[r], rows = a.rb_rows[r];
    // work-list check: the union fits the tables the launch sized
    if (W > a.wmax_union || W < 1 || it.i0 >= rows || it.j0 >= W) {
        if (tid == 0 && a.status) atomicExch(a.status, kDevBadTile);
        return;
    }
    // union-column map, one thread per stored block of the row block
    for (int64_t k = b0 + tid; k < b1; k += blockDim.x) {
        const int c = a.col_idx[k], w = a.cbp[c + 1] - a.cbp[c], ld = a.ld[c], u0 = a.ucol0[k];
        if (u0 < 0 || u0 + w > W) {
            if (a.status) atomicExch(a.status, kDevBadTile);
            continue;
        }
        for (int q = 0; q < w; ++q) {
            sUoff[u0 + q] = a.blk_off[k] + q;
            sUld[u0 + q] = ld;
            sUcol[u0 + q] = a.cbp[c] + q;
        }
    }
    __syncthreads();

    const T alpha = T(a.alpha), gamma = T(a.gamma), beta = T(a.beta);
    const int ty = tid >> 4, tx = tid & 15;       // rows ty*4 .., columns tx*4 ..
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < W; k0 += kKT) {
        // A tile: rows i0 + i, union columns k0 + kk
        for (int e = tid; e < kMT * kKT; e += 256) {
            const int i = e / kKT, kk = e % kKT, u = k0 + kk, row = it.i0 + i;
            T v = T(0);
            if (u < W && row < rows) v = a.A[sUoff[u] + (int64_t)row * sUld[u]];
            sA[i][kk] = v;
        }
        // X tile: X[union k0 + kk][union j0 + jj] (row-major, global column order)
        for (int e = tid; e < kKT * kNT; e += 256) {
            const int kk = e / kNT, jj = e % kNT, u = k0 + kk, v2 = it.j0 + jj;
            T v = T(0);
            if (u < W && v2 < W) v = T(a.X[(int64_t)sUcol[u] * a.n_cols + sUcol[v2]]);
            sX[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKT; ++kk) {
            T av[4], xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = sA[ty * 4 + i][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[j] = sX[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], xv[j], acc[i][j]);
        }
        __syncthreads();
    }

    // ---- C = alpha (A X + gamma A) + beta C ------------------------------------
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = it.i0 + ty * 4 + i;
        if (row >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int u = it.j0 + tx * 4 + j;
            if (u >= W) continue;
            const int64_t o = sUoff[u] + (int64_t)row * sUld[u];
            // in the working precision (FP64 arithmetic runs at 1/64 rate here)
            T v = acc[i][j];
            if (gamma != T(0)) v = fma(gamma, a.A[o], v);
            v *= alpha;
            if (beta != T(0)) v = fma(beta, a.C[o], v);
            a.C[o] = v;
        }
    }
    // padding columns of the row chunk's blocks are written as zero (once)
    if (it.j0 == 0) {
        for (int64_t k = b0; k < b1; ++k) {
            const int c = a.col_idx[k], w = a.cbp[c + 1] - a.cbp[c], ld = a.ld[c];
            const int pad = ld - w;
            if (pad == 0) continue;
            for (int e = tid; e < kMT * pad; e += 256) {
                const int row = it.i0 + e / pad;
                if (row < rows) a.C[a.blk_off[k] + (int64_t)row * ld + w + e % pad] = T(0);
            }
        }
    }
}

// Exact product a b = p + e (e = fma(a, b, -p)) added into the running sum
// (s, comp) with a compensated (two-sum) step: the per-lane block sum keeps
// about twice the working precision, without FP64 arithmetic per entry.
template <typename T>
__device__ __forceinline__ void add_product(T a, T b, T& s, T& comp) {
    const T p = a * b, e = fma(a, b, -p);
    const T t = s + p, bp = t - s;
    comp += (s - (t - bp)) + (p - bp) + e;
    s = t;
}

// tr(D^T G): warps take stored blocks in turn; lanes walk a block's 16-byte
// chunks (the chunk index within a row advances by 32 mod chunks-per-row, no
// division), padding columns masked.  Per lane the block's products are
// summed with the compensated step above and added to an FP64 lane total;
// lane totals are reduced in the warp and the CTA, one atomic per CTA.
template <typename T>
__global__ void __launch_bounds__(256) trace_kernel(const TraceArgs<T> a) {
    constexpr int CH = 16 / sizeof(T);
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    __shared__ double sRed[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double total = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * 8 + wid; k < a.n_blocks; k += (int64_t)gridDim.x * 8) {
        const int r = a.block_rb[k];
        const int c = a.col_idx[k], w = a.cbp[c + 1] - a.cbp[c], ld = a.ld[c];
        const int nq = ld / CH, n = a.rb_rows[r] * nq, step = 32 % nq;
        const V* Dv = reinterpret_cast<const V*>(a.D + a.blk_off[k]);
        const V* Gv = reinterpret_cast<const V*>(a.G + a.blk_off[k]);
        T s = T(0), comp = T(0);
        int q = lane % nq;
        for (int e = lane; e < n; e += 32) {
            const V dv = Dv[e], gv = Gv[e];
            const T* dp = reinterpret_cast<const T*>(&dv);
            const T* gp = reinterpret_cast<const T*>(&gv);
#pragma unroll
            for (int h = 0; h < CH; ++h)
                if (q * CH + h < w) add_product(dp[h], gp[h], s, comp);
            q += step;
            if (q >= nq) q -= nq;
        }
        total += (double)s + (double)comp;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
    if (lane == 0) sRed[wid] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sRed[i];
        if (t != 0.0) atomicAdd(a.out, t);
    }
}

}  // namespace

template <typename T>
size_t mmult_smem_bytes(int wmax_union) {
    return (size_t)wmax_union * (sizeof(int64_t) + 2 * sizeof(int));
}

template <typename T>
cudaError_t launch_mmult(const MmultArgs<T>& a, cudaStream_t s) {
    if (a.n_items == 0) return cudaSuccess;
    const size_t smem = mmult_smem_bytes<T>(a.wmax_union);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mmult_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    mmult_kernel<T><<<(unsigned)a.n_items, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trace(const TraceArgs<T>& a, cudaStream_t s) {
    if (a.n_blocks == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (a.n_blocks + 7) / 8;
    trace_kernel<T><<<(unsigned)std::min<int64_t>(need, 8 * (int64_t)sms), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template size_t mmult_smem_bytes<float>(int);
template size_t mmult_smem_bytes<double>(int);
template cudaError_t launch_mmult<float>(const MmultArgs<float>&, cudaStream_t);
template cudaError_t launch_mmult<double>(const MmultArgs<double>&, cudaStream_t);
template cudaError_t launch_trace<float>(const TraceArgs<float>&, cudaStream_t);
template cudaError_t launch_trace<double>(const TraceArgs<double>&, cudaStream_t);

}  // namespace femf
