// Post-multiplication of an FP32 multivector on the tcgen05 tensor cores
// (Alg. 7, Sec. 3.6; Eqs. G_ops1/G_ops2): C = alpha (A X + gamma A) + beta C
// on C's pattern, A and C sharing it.
//
// Row block r needs only its union columns (the columns of its stored
// blocks, in padded coordinates: every block contributes its row stride ld,
// so every 16-byte chunk of a block row is a chunk of the union): C_r =
// A_r X[union, union].  An item is (row block, 64-row chunk, 128-column
// chunk of the union), as for the SIMT kernel.  The product is taken
// transposed, C^T = X^T A^T: the MMA's M = 128 rows are the item's output
// columns, its N = 64 columns the item's rows, and K runs over the union in
// chunks of 32 (one 128-byte swizzled row of TF32).  The accumulator (128
// lanes x 64 FP32 columns) lives in tensor memory.
//
// Precision: a 3-term TF32 split, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (hi = TF32 rounding, lo = the FP32 remainder): about 2^-21 relative per
// product, inside the FP32 tolerance of C.
//
// Operands.  X + gamma I is transposed, rounded to FP32, split, and laid out
// in padded global coordinates once per call (round_xt_kernel): XT[pv][pu] =
// (X + gamma I)[u][v], zero for padding columns (the gamma term rides on X).  A panel row of X^T (an output column v) over a
// K chunk is then 16-byte copies from one row of XT, straight into the
// swizzled tile (cp.async).  A is read with 16-byte loads, split in
// registers, and stored swizzled.  One 48 KB stage per CTA, so that four
// CTAs share an SM and one's copies overlap another's MMAs and epilogue (two
// stages at two CTAs per SM measured slower); an mbarrier per stage tells
// when its MMAs have completed.
//
// Roles.  All 256 threads stage; thread 0 issues the MMAs (3 per K step of
// 8, 4 K steps per chunk) and commits them; all 8 warps read the
// accumulator back (warp w: tensor-memory lanes 32 (w % 4) .. + 31, item rows
// 32 (w / 4) .. + 31) and write C.  Persistent CTAs, 4 per SM, take items in
// a fixed stride.  Every mbarrier wait is bounded in time; on a time-out the
// kernel sets the status word, waits (bounded) for the MMAs in flight and
// frees its tensor memory.
#include <algorithm>

#include "fe_internal.h"
#include "tc_common.cuh"

namespace femf {
namespace {

constexpr int kTcRows = 64;                          // item rows: N of the MMA
constexpr int kTcCols = 128;                         // item output columns: M of the MMA
constexpr int kTcK = 32;                             // union columns per K chunk
constexpr int kXPanel = kTcCols * 128;               // bytes of an X^T panel (hi or lo)
constexpr int kAPanel = kTcRows * 128;               // bytes of an A^T panel (hi or lo)
constexpr int kTcStage = 2 * kXPanel + 2 * kAPanel;  // 48 KB: hi and lo of both operands
constexpr int kTcStages = 1;                         // one stage: four CTAs per SM overlap instead
constexpr int kTcCtasPerSm = 4;
constexpr int kTcThreads = 256;
constexpr int kTcTmemCols = 64;
constexpr uint64_t kTcWaitNs = 200ull * 1000 * 1000;   // 0.2 s

__device__ __forceinline__ void cp_async16z(uint32_t dst, const void* src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
}

// XT[pv][pu] = (X + gamma I)[pglob[pu]][pglob[pv]] rounded to FP32 and split
// into a TF32 high part and the FP32 remainder; zero where either padded
// column is padding (pglob < 0).  On a row block's union A (X + gamma I) =
// A X + gamma A, so the gamma term needs no second read of A.
__global__ void __launch_bounds__(256) round_xt_kernel(const double* __restrict__ X, const int32_t* __restrict__ pglob,
                                                       int n_pcols, int n_cols, double gamma, float* __restrict__ xt_hi,
                                                       float* __restrict__ xt_lo) {
    const int64_t total = (int64_t)n_pcols * n_pcols;
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256) {
        const int pv = (int)(i / n_pcols), pu = (int)(i - (int64_t)pv * n_pcols);
        const int gu = pglob[pu], gv = pglob[pv];
        const float x =
            (gu >= 0 && gv >= 0) ? (float)(X[(int64_t)gu * n_cols + gv] + (gu == gv ? gamma : 0.0)) : 0.f;
        const float h = tf32_hi(x);
        xt_hi[i] = h;
        xt_lo[i] = x - h;
    }
}

__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm) mmult_tc_kernel(const MmultArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    unsigned char* ring = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);   // stages, 1 KB aligned
    int64_t* sUoff = reinterpret_cast<int64_t*>(ring + kTcStages * kTcStage);   // [W] offset of union column u at row 0
    int* sUld = reinterpret_cast<int*>(sUoff + a.wmax_union);             // [W] row stride
    int* sUcol = sUld + a.wmax_union;                                      // [W] global column, -1 = padding
    int* sUpg = sUcol + a.wmax_union;                                      // [W] padded global column
    __shared__ __align__(8) uint64_t bDone[kTcStages];
    __shared__ uint32_t sTmem;
    __shared__ volatile int sFail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bDone[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sFail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTmem)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sTmem;

    int chunk_no = 0;                         // K chunks this CTA has staged: stage chunk_no % kTcStages
    uint32_t last_bar = 0, last_parity = 0;   // thread 0: the latest commit
    bool issued = false;
    const uint32_t idesc = tf32_idesc(kTcCols, kTcRows);
    // the next item's record and row-block data are fetched while the
    // current item runs
    struct RowInfo {
        MmultItem it;
        int64_t b0, b1;
        int W, rows;
    };
    auto row_info = [&](int64_t item) {
        RowInfo ri;
        ri.it = a.items[item];
        ri.b0 = a.row_ptr[ri.it.r];
        ri.b1 = a.row_ptr[ri.it.r + 1];
        ri.W = a.rb_union[ri.it.r];
        ri.rows = a.rb_rows[ri.it.r];
        return ri;
    };
    RowInfo nxt{};
    if (blockIdx.x < a.n_items) nxt = row_info(blockIdx.x);
    for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const RowInfo cur = nxt;
        if (item + gridDim.x < a.n_items) nxt = row_info(item + gridDim.x);
        const MmultItem it = cur.it;
        const int64_t b0 = cur.b0, b1 = cur.b1;
        const int W = cur.W, rows = cur.rows;
        // work-list check: the padded union fits the tables the launch sized
        if (W > a.wmax_union || W < 1 || it.i0 >= rows || it.j0 >= W) {
            if (tid == 0 && a.status) atomicExch(a.status, kDevBadTile);
            continue;
        }
        __syncthreads();                          // the previous item's tables are done with
        // union-column map, one thread per (stored block, 4-column chunk)
        for (int64_t e = b0 * 4 + tid; e < b1 * 4; e += blockDim.x) {
            const MmBlock bk = a.mm_blocks[e >> 2];
            const int q0 = 4 * (int)(e & 3);
            if (bk.u0 < 0 || bk.u0 + bk.ld > W || bk.u0 % 4 != 0 || bk.ld > 16) {
                if (a.status) atomicExch(a.status, kDevBadTile);
                continue;
            }
            for (int q = q0; q < q0 + 4 && q < bk.ld; ++q) {
                sUoff[bk.u0 + q] = bk.off + q;
                sUld[bk.u0 + q] = bk.ld;
                sUcol[bk.u0 + q] = q < bk.w ? bk.gcol0 + q : -1;
                sUpg[bk.u0 + q] = bk.pcol0 + q;
            }
        }
        __syncthreads();

        const int nk = (W + kTcK - 1) / kTcK;
        for (int t = 0; t < nk; ++t, ++chunk_no) {
            const int stage = chunk_no % kTcStages, use = chunk_no / kTcStages;
            // the stage is free once the MMAs of its previous use have completed
            if (tid == 0 && use > 0 && !mbar_wait(smem_u32(&bDone[stage]), (uint32_t)((use - 1) & 1), kTcWaitNs))
                sFail = 1;
            __syncthreads();
            if (sFail) break;
            unsigned char* xh = ring + stage * kTcStage;
            unsigned char* xl = xh + kXPanel;
            unsigned char* ah = xl + kXPanel;
            unsigned char* al = ah + kAPanel;
            const int k0 = t * kTcK;
            // X^T: operand row m = output union column j0 + m; 16-byte chunk j =
            // union columns k0 + 4j .. + 3, one row of XT in padded coordinates
            for (int e = tid; e < kTcCols * 8; e += kTcThreads) {
                const int m = e >> 3, j = e & 7;
                const int uo = it.j0 + m, uk = k0 + 4 * j;
                const bool ok = uo < W && uk < W;
                const int64_t o = ok ? (int64_t)sUpg[uo] * a.n_pcols + sUpg[uk] : 0;
                cp_async16z(smem_u32(xh + sw_off(m, j)), a.XThi + o, ok);
                cp_async16z(smem_u32(xl + sw_off(m, j)), a.XTlo + o, ok);
            }
            // A^T: operand row n = item row i0 + n, the same union chunks, split
            for (int e = tid; e < kTcRows * 8; e += kTcThreads) {
                const int n = e >> 3, j = e & 7;
                const int row = it.i0 + n, uk = k0 + 4 * j;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row < rows && uk < W)
                    v = __ldg(reinterpret_cast<const float4*>(a.A + sUoff[uk] + (int64_t)row * sUld[uk]));
                const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
                *reinterpret_cast<float4*>(ah + sw_off(n, j)) = h;
                *reinterpret_cast<float4*>(al + sw_off(n, j)) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t xh0 = smem_u32(xh), xl0 = smem_u32(xl), ah0 = smem_u32(ah), al0 = smem_u32(al);
#pragma unroll
                for (int kk = 0; kk < kTcK / 8; ++kk) {
                    // the item's first product starts the sum
                    mma_tf32(tmem, sw128_desc(xh0 + 32 * kk), sw128_desc(ah0 + 32 * kk), idesc, (t > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(tmem, sw128_desc(xh0 + 32 * kk), sw128_desc(al0 + 32 * kk), idesc, 1u);
                    mma_tf32(tmem, sw128_desc(xl0 + 32 * kk), sw128_desc(ah0 + 32 * kk), idesc, 1u);
                }
                mma_commit(smem_u32(&bDone[stage]));
                last_bar = smem_u32(&bDone[stage]);
                last_parity = (uint32_t)(use & 1);
                issued = true;
            }
        }
        if (sFail) break;
        // the item's last commit covers all of its MMAs
        if (tid == 0 && !mbar_wait(last_bar, last_parity, kTcWaitNs)) sFail = 1;
        __syncthreads();
        if (sFail) break;
        tc_fence_after();

        // ---- C = alpha A (X + gamma I) + beta C; padding columns written as zero --
        const int q = warp & 3, h = warp >> 2;
        const int uo = it.j0 + 32 * q + lane;     // this thread's output union column
        const float alpha = (float)a.alpha, beta = (float)a.beta;
        const bool col_ok = uo < W;
        const int64_t ou = col_ok ? sUoff[uo] : 0;
        const int ldu = col_ok ? sUld[uo] : 0;
        const bool pad = !col_ok || sUcol[uo] < 0;
        // 16 rows of accumulator columns at a time (a warp-wide load); then, 8
        // rows at a time, all the loads of C before the stores, so that the
        // loads are not held behind the stores to the same array
#pragma unroll
        for (int i0 = 0; i0 < 32; i0 += 16) {
            float acc[16];
            tmem_load<16>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h + i0), acc);
            if (col_ok) {
#pragma unroll
                for (int i1 = 0; i1 < 16; i1 += 8) {
                    const int row0 = it.i0 + 32 * h + i0 + i1;
                    float* c0 = a.C + ou + (int64_t)row0 * ldu;
                    float cv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        cv[i] = (beta != 0.f && !pad && row0 + i < rows) ? c0[(int64_t)i * ldu] : 0.f;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (row0 + i < rows) c0[(int64_t)i * ldu] = pad ? 0.f : fmaf(beta, cv[i], alpha * acc[i1 + i]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();                          // the accumulator is read before the next item's MMAs
    }

    if (sFail) {
        if (tid == 0) {
            if (a.status) atomicExch(a.status, kDevTimeout);
            if (issued) mbar_wait(last_bar, last_parity, kTcWaitNs);   // the MMAs in flight
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    }
}

}  // namespace

size_t mmult_tc_smem_bytes(int wmax_union) {
    return 1024 + (size_t)kTcStages * kTcStage + (size_t)wmax_union * (sizeof(int64_t) + 3 * sizeof(int));
}

cudaError_t launch_mmult_tc(const MmultArgs<float>& a, float* xt, cudaStream_t s) {
    if (a.n_items == 0) return cudaSuccess;
    const size_t smem = mmult_tc_smem_bytes(a.wmax_union);
    if (smem > kMmultTcSmemMax) return cudaErrorInvalidValue;
    MmultArgs<float> b = a;
    const int64_t n = (int64_t)a.n_pcols * a.n_pcols;
    b.XThi = xt;
    b.XTlo = xt + n;
    round_xt_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 2048), 256, 0, s>>>(a.X, a.pglob, a.n_pcols,
                                                                                     a.n_cols, a.gamma, xt, xt + n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(mmult_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmultTcSmemMax);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int sms = usable_sms(a.sm_limit);
    if (sms < 1) return cudaErrorInvalidDevice;
    const unsigned grid = (unsigned)std::min<int64_t>(a.n_items, kTcCtasPerSm * (int64_t)sms);
    mmult_tc_kernel<<<grid, kTcThreads, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace femf
