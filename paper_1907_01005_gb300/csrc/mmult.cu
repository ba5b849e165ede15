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
// The union is taken in padded coordinates (each stored block contributes
// its row stride ld, so every 16-byte chunk of a block row is one chunk of
// the union); padding columns meet zero rows of X and are written as zero.
// X is first rounded to the working precision once per call (FP32: into a
// region of C's table buffer).  Work item: (row block, 64-row chunk,
// 128-column chunk of the padded union).  256 threads; warp w owns a 32 x 32
// sub-tile (rows 32 (w / 4), columns 32 (w % 4)) and skips the product when
// its columns lie beyond the union; lane l owns rows l / 4 + 8 i (i < 4) and
// columns 8 (l % 4) + j (j < 8) of it.  The union is walked in k-tiles
// staged by cp.async (16-byte chunks of A, element copies of X) into two
// shared-memory buffers, so the copies of tile t + 1 overlap the FMAs of t.
#include <algorithm>
#include <type_traits>

#include "fe_internal.h"

namespace femf {
namespace {

constexpr int kMT = 64;          // rows per tile
constexpr int kNT = 128;         // output columns per tile

template <typename T>
struct MmGeo {
    static constexpr int KT = sizeof(T) == 4 ? 32 : 16;   // union columns per k-tile
    static constexpr int CH = 16 / sizeof(T);              // elements per 16-byte chunk
    static constexpr int LDA = KT + 4;                     // row stride of the A tile (16-byte multiple)
    static constexpr int LDX = kNT + 4;                    // row stride of the X tile
    static constexpr int STAGE = kMT * LDA + KT * LDX;     // elements of one buffer
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 16 : 0) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0) : "memory");
}

// resident CTAs per SM the register budget must allow (32 accumulators a thread)
template <typename T>
constexpr int kMmMinBlocks = sizeof(T) == 4 ? 3 : 2;

template <typename T>
__global__ void __launch_bounds__(256, kMmMinBlocks<T>) mmult_kernel(const MmultArgs<T> a) {
    using G = MmGeo<T>;
    constexpr int KT = G::KT, CH = G::CH, LDA = G::LDA, LDX = G::LDX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* stage = reinterpret_cast<T*>(smem_raw);                                   // 2 x [A tile | X tile]
    int64_t* sUoff = reinterpret_cast<int64_t*>(stage + 2 * G::STAGE);          // [Wp] offset of column u at row 0
    int* sUld = reinterpret_cast<int*>(sUoff + a.wmax_union);                   // [Wp] row stride
    int* sUcol = sUld + a.wmax_union;                                            // [Wp] global column, -1 = padding

    const MmultItem it = a.items[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = it.r;
    const int64_t b0 = a.row_ptr[r], b1 = a.row_ptr[r + 1];
    const int W = a.rb_union[r], rows = a.rb_rows[r];
    // work-list check: the padded union fits the tables the launch sized
    if (W > a.wmax_union || W < 1 || it.i0 >= rows || it.j0 >= W) {
        if (tid == 0 && a.status) atomicExch(a.status, kDevBadTile);
        return;
    }
    // union-column map, one thread per stored block of the row block
    for (int64_t k = b0 + tid; k < b1; k += blockDim.x) {
        const int c = a.col_idx[k], w = a.cbp[c + 1] - a.cbp[c], ld = a.ld[c], u0 = a.ucol0[k];
        if (u0 < 0 || u0 + ld > W || u0 % CH != 0) {
            if (a.status) atomicExch(a.status, kDevBadTile);
            continue;
        }
        for (int q = 0; q < ld; ++q) {
            sUoff[u0 + q] = a.blk_off[k] + q;
            sUld[u0 + q] = ld;
            sUcol[u0 + q] = q < w ? a.cbp[c] + q : -1;
        }
    }
    __syncthreads();

    const int nk = (W + KT - 1) / KT;
    auto load_tile = [&](int t, int buf) {
        T* sA = stage + buf * G::STAGE;
        T* sX = sA + kMT * LDA;
        const int k0 = t * KT;
        // A: 64 rows x KT union columns in 16-byte chunks
        for (int e = tid; e < kMT * (KT / CH); e += 256) {
            const int i = e / (KT / CH), cc = e % (KT / CH), u = k0 + cc * CH, row = it.i0 + i;
            const bool ok = u < W && row < rows;
            const T* src = ok ? a.A + sUoff[u] + (int64_t)row * sUld[u] : a.A;
            cp_async16(sA + i * LDA + cc * CH, src, ok);
        }
        // X: KT union rows x 128 union columns (zero for padding and beyond the union)
        for (int e = tid; e < KT * kNT; e += 256) {
            const int kk = e / kNT, jj = e % kNT, u = k0 + kk, v = it.j0 + jj;
            const int gu = u < W ? sUcol[u] : -1, gv = v < W ? sUcol[v] : -1;
            const bool ok = gu >= 0 && gv >= 0;
            cp_async_elem(sX + kk * LDX + jj, ok ? a.Xw + (int64_t)gu * a.n_cols + gv : a.Xw, ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    const int wr = (warp >> 2) * 32, wc = (warp & 3) * 32;
    const int lr = lane >> 2, lc = (lane & 3) * 8;
    const bool busy = it.j0 + wc < W;             // warp-uniform: columns of this warp in the union
    T acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);

    load_tile(0, 0);
    for (int t = 0; t < nk; ++t) {
        if (t + 1 < nk) load_tile(t + 1, (t + 1) & 1);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        if (busy) {
            const T* sA = stage + (t & 1) * G::STAGE;
            const T* sX = sA + kMT * LDA;
#pragma unroll 4
            for (int kk = 0; kk < KT; ++kk) {
                T av[4], xv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = sA[(wr + lr + 8 * i) * LDA + kk];
                if constexpr (sizeof(T) == 4) {
                    const float4 x0 = *reinterpret_cast<const float4*>(sX + kk * LDX + wc + lc);
                    const float4 x1 = *reinterpret_cast<const float4*>(sX + kk * LDX + wc + lc + 4);
                    xv[0] = x0.x; xv[1] = x0.y; xv[2] = x0.z; xv[3] = x0.w;
                    xv[4] = x1.x; xv[5] = x1.y; xv[6] = x1.z; xv[7] = x1.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 8; j += 2) {
                        const double2 x = *reinterpret_cast<const double2*>(sX + kk * LDX + wc + lc + j);
                        xv[j] = x.x; xv[j + 1] = x.y;
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], xv[j], acc[i][j]);
            }
        }
        __syncthreads();                              // buffer t & 1 is refilled at t + 2
    }

    // ---- C = alpha (A X + gamma A) + beta C; padding columns written as zero --
    if (!busy) return;
    const T alpha = T(a.alpha), gamma = T(a.gamma), beta = T(a.beta);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = it.i0 + wr + lr + 8 * i;
        if (row >= rows) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int u = it.j0 + wc + lc + j;
            if (u >= W) continue;
            const int64_t o = sUoff[u] + (int64_t)row * sUld[u];
            if (sUcol[u] < 0) {
                a.C[o] = T(0);
                continue;
            }
            // in the working precision (FP64 arithmetic runs at 1/64 rate here)
            T v = acc[i][j];
            if (gamma != T(0)) v = fma(gamma, a.A[o], v);
            v *= alpha;
            if (beta != T(0)) v = fma(beta, a.C[o], v);
            a.C[o] = v;
        }
    }
}

// X rounded to FP32 once per call
__global__ void __launch_bounds__(256) round_x_kernel(const double* X, float* Xw, int64_t n) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) Xw[i] = float(X[i]);
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
    return (size_t)2 * MmGeo<T>::STAGE * sizeof(T) + (size_t)wmax_union * (sizeof(int64_t) + 2 * sizeof(int));
}

template <typename T>
cudaError_t launch_mmult(const MmultArgs<T>& a, float* x_round, cudaStream_t s) {
    if (a.n_items == 0) return cudaSuccess;
    MmultArgs<T> b = a;
    if constexpr (sizeof(T) == 4) {
        const int64_t n = (int64_t)a.n_cols * a.n_cols;
        round_x_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(a.X, x_round, n);
        b.Xw = x_round;
    } else {
        b.Xw = a.X;
    }
    const size_t smem = mmult_smem_bytes<T>(a.wmax_union);
    if (smem > kMmultSmemMax) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mmult_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmultSmemMax);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    mmult_kernel<T><<<(unsigned)a.n_items, 256, smem, s>>>(b);
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
template cudaError_t launch_mmult<float>(const MmultArgs<float>&, float*, cudaStream_t);
template cudaError_t launch_mmult<double>(const MmultArgs<double>&, float*, cudaStream_t);
template cudaError_t launch_trace<float>(const TraceArgs<float>&, cudaStream_t);
template cudaError_t launch_trace<double>(const TraceArgs<double>&, cudaStream_t);

}  // namespace femf
