// Gram products of FP32 multivectors on the tcgen05 tensor cores with an
// error-free split (C = A^T B over stored blocks, Alg. 8; FP64-accurate
// result).
//
// Numerics.  Rows are taken in windows of at most KX rows.  In a window every
// FP32 value x of union column m is normalised by the window's power-of-two
// bound 2^E (|x| < 2^E, E per column and window) and written as a sum of
// bf16 slices y_s (every slice exact in bf16, every slice product exact in
// FP32):
//   P^T P  five slices on fixed grids, y_s = q_s 2^(-8 s), |q_1| <= 256,
//          |q_s| <= 128 for s >= 2; products with s + t <= 6 are kept;
//   P^T Y  y_1 = q_1 2^-8 on the fixed grid, y_2, y_3 the bf16 roundings of
//          the remainders ("natural" slices); products with s + t <= 4.
// The product of slices s and t has level L = s + t.  The tensor cores sum
// each level class of a window in an FP32 accumulator in tensor memory:
//   P^T P  levels 2, 3 and 4 each on its own: their window sums are integers
//          (units 2^-16, 2^-24, 2^-32) below 2^24 for KX = 192 rows, hence
//          exact whatever the rounding of the tensor-core adder; levels 5 and
//          6 together, below 2^-24 of the result per row, so their FP32
//          rounding is immaterial;
//   P^T Y  level 2 exact (KX = 256 rows), levels 3 and 4 together.
// After each window the class sums are converted to integers in units of
// 2^-(8 LMAX) and added into an int64 per output element, scaled by
// 2^(E_m(w) + E_n(w)) relative to a running per-column reference exponent R
// (the largest window exponent so far): the accumulator is shifted right when
// R grows, the window value when its exponents are below R.  The int64 is
// converted to FP64 with integer operations only (the FP64 pipe of this GPU
// is slow) and added into the dense FP64 result with one atomic per element.
//
// Work item: (group of consecutive row blocks, 128 x 128 tile (mi, ni) of the
// group's union columns, range of the group's rows).  Operand A of the MMA is
// the panel of the tile's 128 A columns (M = 128 rows of the MMA, one per
// union column, K = rows of the multivector), operand B the panel of its
// N <= 128 B columns; D[m][n] = sum_k A[m][k] B[n][k] lands in tensor-memory
// lane m, column n (+ 128 per level class).  Panels are staged 64 rows at a
// time as bf16 slices in the K-major layout with the 128-byte swizzle (an
// operand row is 64 bf16 = 128 bytes), into one of two buffers, so that the
// slicing of chunk c+1 overlaps the MMAs of chunk c.  One thread issues the
// tcgen05.mma instructions and commits them to the buffer's mbarrier; all
// sixteen warps stage, and all sixteen read the accumulators back
// (tcgen05.ld: warp w reaches lanes 32 (w % 4) .. + 31 and takes 32 of the
// tile's columns).  Every wait on an mbarrier is bounded in time; on a
// time-out the kernel sets the status word, waits (bounded) for the MMAs in
// flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "fe_internal.h"

namespace femf {
namespace {

constexpr int kST = 128;                  // output tile edge in union columns (M of the MMA, N <= kST)
constexpr int kThreads = 512;             // 16 warps
constexpr int kKC = 64;                   // rows of a staged chunk: 64 bf16 = one 128-byte swizzle row
constexpr int kPanel = kST * 128;         // bytes of one slice panel (128 operand rows of 128 bytes)
constexpr int kBuf = 96 * 1024;           // bytes of one staging buffer (both operands of a chunk)
constexpr int kSmemDyn = 2 * kBuf + 1024; // two buffers + slack for the 1024-byte alignment
constexpr int kNone = -30000;             // exponent of an all-zero column
constexpr int kMaxRows = (2 * kMaxP + 1) * (2 * kMaxP + 1) * (2 * kMaxP + 1);   // rows of a row block
constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;   // bounded mbarrier waits (0.2 s)

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand, rows of 128 bytes with the
// 128-byte swizzle, 8-row groups 1024 bytes apart (stride byte offset); the
// leading byte offset is unused for this layout (one swizzle atom along K).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (16 B, unused)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Waits until the barrier's phase `parity` has completed, for at most
// `limit_ns`; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// 32 lanes x 8 consecutive FP32 columns of tensor memory: thread i of the
// warp receives lane (32 (warp % 4) + i), columns col .. col + 7.  The wait
// is tied to the destination registers so that no use moves above it.
__device__ __forceinline__ void tmem_load8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- numerics helpers ------------------------------------------------------------
// t * 2^e2 as a double, from integer operations only (round to nearest even)
__device__ __forceinline__ double i64_scaled_to_double(long long t, int e2) {
    if (t == 0) return 0.0;
    const unsigned long long sign = t < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
    int msb = 63 - __clzll(a);
    unsigned long long mant;
    if (msb <= 52) {
        mant = a << (52 - msb);
    } else {
        const int sh = msb - 52;
        const unsigned long long rem = a & ((1ull << sh) - 1);
        const unsigned long long half = 1ull << (sh - 1);
        mant = a >> sh;
        if (rem > half || (rem == half && (mant & 1ull))) {
            mant += 1;
            if (mant >> 53) {
                mant >>= 1;
                msb += 1;
            }
        }
    }
    const long long be = (long long)msb + e2 + 1023;
    if (be <= 0) return 0.0;
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }   // |e| <= 126

// Rounds v 2^U (|v 2^U| < 2^62, v a float) to an int64 with two 32-bit
// conversions (the 64-bit one runs on the FP64 pipe): the high part on the
// 2^-H grid, then the exact remainder.
template <int U, int H>
__device__ __forceinline__ long long round_scaled_i64(float v) {
    const float hi = rintf(v * pow2f(H));
    const float rem = fmaf(-hi, pow2f(-H), v);               // exact
    return ((long long)(int)hi << (U - H)) + (long long)__float2int_rn(rem * pow2f(U));
}

// Loads rows kstart .. kstart+7 of the group (those at or past kend read as
// zero) of one union column into v and returns max |x|.  Consecutive rows of
// a row block are ld elements apart.  When the 8 rows touch at most two row
// blocks (always for p >= 2, whose row blocks hold at least 64 rows) the
// addresses come from two bases and all loads are independent; otherwise the
// rows are walked one by one.
__device__ __forceinline__ float load8(const float* __restrict__ X, int ci, const int64_t* sOff, int n_u,
                                       const int* sPref, int nrb, int kstart, int kend, float (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (ci < 0 || kstart >= kend) return 0.f;
    const int slot = ci >> 16, a = (ci >> 8) & 0xff, ld = ci & 0xff;
    int r = 0;
    while (r < nrb - 1 && kstart >= sPref[r + 1]) ++r;
    const int end_r = sPref[r + 1];
    if (r + 1 >= nrb || sPref[r + 2] >= kstart + 8) {
        const int64_t o0 = sOff[r * n_u + slot];
        const int64_t o1 = r + 1 < nrb ? sOff[(r + 1) * n_u + slot] : -1;
        const int64_t b0 = o0 + (int64_t)(kstart - sPref[r]) * ld + a;   // row kstart + i -> b0 + i ld
        const int64_t b1 = o1 + a - (int64_t)end_r * ld;                  // row k >= end_r -> b1 + k ld
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = kstart + i;
            const bool in0 = k < end_r;
            const bool ok = k < kend && (in0 ? o0 >= 0 : o1 >= 0);
            const int64_t ix = in0 ? b0 + (int64_t)i * ld : b1 + (int64_t)k * ld;
            if (ok) v[i] = __ldg(X + ix);
        }
    } else {
        int rr = r, e = end_r;
        int64_t o = sOff[rr * n_u + slot];
        int64_t idx = o + (int64_t)(kstart - sPref[rr]) * ld + a;
        for (int i = 0; i < 8; ++i) {
            const int k = kstart + i;
            if (k >= kend) break;
            if (k == e) {                     // first row of the next row block (k < kend <= sPref[nrb])
                ++rr;
                e = sPref[rr + 1];
                o = sOff[rr * n_u + slot];
                idx = o + a;
            }
            if (o >= 0) v[i] = __ldg(X + idx);
            idx += ld;
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(v[i]));
    return mx;
}

// Byte offset of 16-byte chunk j (rows 8j .. 8j+7 of the chunk) of operand
// row c in a slice panel: the 128-byte swizzle (chunk index XOR row mod 8)
__device__ __forceinline__ uint32_t sw_off(int c, int j) { return (uint32_t)(c * 128 + ((j ^ (c & 7)) << 4)); }

// Slices 8 values (already multiplied by f1) of operand row c into S bf16
// slices y_s = q_s 2^(-8 s) on fixed grids, one 16-byte chunk per slice panel.
template <int S>
__device__ __forceinline__ void slice_store(unsigned char* base, int c, int j, float f2, const float (&v)[8]) {
    float r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = v[i] * f2;
    const uint32_t off = sw_off(c, j);
#pragma unroll
    for (int s = 1; s <= S; ++s) {
        const float up = pow2f(8 * s), dn = pow2f(-8 * s);
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float q0 = rintf(r[2 * i] * up), q1 = rintf(r[2 * i + 1] * up);
            r[2 * i] = fmaf(-q0, dn, r[2 * i]);
            r[2 * i + 1] = fmaf(-q1, dn, r[2 * i + 1]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(q0 * dn, q1 * dn);   // exact
            w[i] = *reinterpret_cast<const uint32_t*>(&b);
        }
        *reinterpret_cast<uint4*>(base + (s - 1) * kPanel + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Three slices with only the first on a fixed grid: y1 = q 2^-8 (|q| <= 256),
// y2 = bf16(x - y1), y3 = bf16(x - y1 - y2).
__device__ __forceinline__ void slice_store_nat(unsigned char* base, int c, int j, float f2, const float (&v)[8]) {
    const uint32_t off = sw_off(c, j);
    uint32_t w1[4], w2[4], w3[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float r0 = v[2 * i] * f2, r1 = v[2 * i + 1] * f2;
        const float q0 = rintf(r0 * 256.f), q1 = rintf(r1 * 256.f);
        r0 = fmaf(-q0, 0.00390625f, r0);
        r1 = fmaf(-q1, 0.00390625f, r1);
        const __nv_bfloat162 b1 = __floats2bfloat162_rn(q0 * 0.00390625f, q1 * 0.00390625f);   // exact
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0, r1);
        r0 -= __low2float(b2);
        r1 -= __high2float(b2);
        const __nv_bfloat162 b3 = __floats2bfloat162_rn(r0, r1);
        w1[i] = *reinterpret_cast<const uint32_t*>(&b1);
        w2[i] = *reinterpret_cast<const uint32_t*>(&b2);
        w3[i] = *reinterpret_cast<const uint32_t*>(&b3);
    }
    *reinterpret_cast<uint4*>(base + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(base + kPanel + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    *reinterpret_cast<uint4*>(base + 2 * kPanel + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
}

// Level class of the product of slices s and t
template <int NCLS>
__host__ __device__ constexpr int level_class(int L) {
    return NCLS == 4 ? (L <= 4 ? L - 2 : 3) : (L == 2 ? 0 : 1);
}

// The window value of one output element from its class sums, as an integer
// in units of 2^-(8 LMAX) of 2^(E_m + E_n)
template <int NCLS>
__device__ __forceinline__ long long window_value(const float (&c)[NCLS]) {
    if constexpr (NCLS == 4) {   // P^T P, units 2^-48
        const int i2 = __float2int_rn(c[0] * pow2f(16));
        const int i3 = __float2int_rn(c[1] * pow2f(24));
        const int i4 = __float2int_rn(c[2] * pow2f(32));
        return ((long long)i2 << 32) + ((long long)i3 << 24) + ((long long)i4 << 16) + round_scaled_i64<48, 32>(c[3]);
    } else {                     // P^T Y, units 2^-32
        const int i2 = __float2int_rn(c[0] * pow2f(16));
        return ((long long)i2 << 16) + round_scaled_i64<32, 16>(c[1]);
    }
}

template <int SA, int SB, int LMAX, int NCLS, bool SYM, bool SAME, int KX, bool NAT>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(const GramTcArgs g) {
    static_assert(KX % kKC == 0, "windows are whole chunks");
    static_assert(!NAT || (SA == 3 && SB == 3), "natural slices: three per operand");
    static_assert(NCLS * kST <= 512, "tensor memory: 128 columns per level class");
    constexpr int TMEM_COLS = NCLS * kST;       // 256 or 512 (a power of two)
    constexpr int U = 8 * LMAX;                 // the flush works in units of 2^-U
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    unsigned char* sm = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
    __shared__ int64_t sOff[kMaxGroup * kMaxUnion];
    __shared__ int sCol[2][kST], sGcol[2][kST];
    __shared__ int sPref[kMaxGroup + 1];
    __shared__ unsigned sMax[2][kST];
    __shared__ int sR[2][kST], sDR[2][kST], sDW[2][kST];
    __shared__ float sF1[2][kST], sF2[2][kST];
    __shared__ __align__(8) uint64_t sBar[2];
    __shared__ uint32_t sTmem;
    __shared__ int sFail;

    const int tid = threadIdx.x, warp = tid >> 5;
    const GramTcItem it = g.items[blockIdx.x];
    const GramTcGroup gr = g.groups[it.group];
    const int mi = it.tile & 0xffff, ni = it.tile >> 16;
    const int nrb = gr.r1 - gr.r0;
    // Work-list check: a group has 1..kMaxGroup row blocks of at most kMaxRows
    // rows and 1..kMaxUnion union column blocks (the shared tables depend on
    // it); a malformed item sets the status word and leaves G untouched.
    if (nrb < 1 || nrb > kMaxGroup || gr.n_u < 1 || gr.n_u > kMaxUnion || gr.width < 1 ||
        gr.width > kMaxUnion * kMaxW || gr.k_rows > kMaxGroup * kMaxRows || mi * kST >= gr.width ||
        ni * kST >= gr.width || (SYM && mi > ni) || it.k0 < 0 || it.k1 > gr.k_rows || it.k0 >= it.k1) {
        if (tid == 0 && g.status) atomicExch(g.status, kDevBadTile);
        return;
    }
    const bool diag = SYM && mi == ni;          // diagonal tile of a symmetric product
    const bool share = SAME && mi == ni;        // ... whose B columns are A's own (B = A)
    const int wa = min(kST, gr.width - mi * kST);          // A columns of the tile
    const int wb = min(kST, gr.width - ni * kST);          // B columns of the tile
    const int N = (wb + 15) & ~15;                         // MMA N (multiple of 16, <= 128)
    // staging buffers: both operands of a chunk in one 96 KB buffer (two
    // buffers, chunks alternate), or for P^T P off-diagonal tiles (160 KB)
    // one buffer spanning both
    constexpr int bytesA = SA * kPanel, bytesB = SB * kPanel;
    const int nbuf = (share ? bytesA : bytesA + bytesB) <= kBuf ? 2 : 1;

    // ---- group tables, tensor memory, barriers ------------------------------------
    for (int e = tid; e < nrb * gr.n_u; e += kThreads) sOff[e] = g.union_off[gr.u_base + e];
    if (tid < kST) {
        const int ma = mi * kST + tid, nb = ni * kST + tid;
        sCol[0][tid] = tid < wa ? g.col_info[gr.c_base + ma] : -1;
        sGcol[0][tid] = tid < wa ? g.col_glob[gr.c_base + ma] : -1;
        sCol[1][tid] = tid < wb ? g.col_info[gr.c_base + nb] : -1;
        sGcol[1][tid] = tid < wb ? g.col_glob[gr.c_base + nb] : -1;
        sR[0][tid] = sR[1][tid] = kNone;
    }
    if (tid == 0) {
        sPref[0] = 0;
        for (int r = 0; r < nrb; ++r) sPref[r + 1] = sPref[r] + g.rows[gr.r0 + r];
        sFail = 0;
        for (int b = 0; b < 2; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sBar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sTmem;
    const bool tables_ok = sPref[nrb] == gr.k_rows;   // the row walk relies on it
    if (!tables_ok && tid == 0 && g.status) atomicExch(g.status, kDevBadTile);

    // this thread's share of the read-back: tensor-memory lane m (operand-A
    // column), columns [32 q, 32 q + 32) of the tile
    const int m = 32 * (warp & 3) + (tid & 31);
    const int q = warp >> 2;
    // warps whose columns lie wholly below the diagonal of a diagonal tile,
    // or beyond the tile's B columns, have nothing to read back
    const bool flush_act = 32 * q < N && !(diag && 32 * q + 31 < 32 * (warp & 3));
    long long acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0;

    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    int chunk_no = 0;
    const uint32_t idesc = bf16_idesc(128, N);

    for (int w0 = it.k0; tables_ok && w0 < it.k1; w0 += KX) {
        const int w1 = min(it.k1, w0 + KX);
        // ---- pass 1: column bounds of the window ----------------------------------
        if (tid < kST) sMax[0][tid] = sMax[1][tid] = 0u;
        __syncthreads();
        {
            const int nchunks8 = (w1 - w0 + 7) >> 3;
            for (int side = 0; side < (share ? 1 : 2); ++side) {
                const int wc = side ? wb : wa;
                const float* X = side ? g.B : g.A;
                for (int t = tid; t < wc * nchunks8; t += kThreads) {
                    const int c = t % wc, j = t / wc;
                    float v[8];
                    const float mx = load8(X, sCol[side][c], sOff, gr.n_u, sPref, nrb, w0 + 8 * j, w1, v);
                    if (mx > 0.f) atomicMax(&sMax[side][c], __float_as_uint(mx));
                }
            }
        }
        __syncthreads();
        // window exponents and the update of the running references
        if (tid < 2 * kST) {
            const int side = tid / kST, c = tid % kST;
            if (side == 0 || !share) {
                const float mx = __uint_as_float(sMax[side][c]);
                const int E = mx > 0.f ? ilogbf(mx) + 1 : kNone;
                const int R = sR[side][c];
                const int newR = E > R ? E : R;
                sDR[side][c] = (R == kNone) ? 0 : min(newR - R, 63);
                sDW[side][c] = (E == kNone) ? 63 : min(newR - E, 63);
                sR[side][c] = newR;
                const int e = (E == kNone) ? 0 : E;
                sF1[side][c] = pow2f(-(e >> 1));
                sF2[side][c] = pow2f(-(e - (e >> 1)));
            }
        }
        __syncthreads();

        // ---- pass 2: chunks of 64 rows, sliced into the staging buffers, MMAs ----
        bool first = true;
        for (int c0 = w0; c0 < w1; c0 += kKC, ++chunk_no) {
            const int b = nbuf == 2 ? (chunk_no & 1) : 0;
            // the buffer is free once the MMAs of its previous chunk are done
            if (pending[b]) {
                if (tid == 0 && !mbar_wait(smem_u32(&sBar[b]), phase[b], kWaitLimitNs)) sFail = 1;
                phase[b] ^= 1u;
                pending[b] = false;
                __syncthreads();
                if (sFail) break;
            }
            unsigned char* bufA = sm + b * kBuf;
            unsigned char* bufB = share ? bufA : bufA + bytesA;
            const int c1 = min(w1, c0 + kKC);
            for (int side = 0; side < (share ? 1 : 2); ++side) {
                const int wc = side ? wb : wa;
                const int wpad = side ? N : wa;          // B rows up to N are read by the MMA
                const float* X = side ? g.B : g.A;
                unsigned char* base = side ? bufB : bufA;
                for (int t = tid; t < wpad * 8; t += kThreads) {
                    const int c = t % wpad, j = t / wpad;
                    float v[8];
                    const int ci = c < wc ? sCol[side][c] : -1;
                    load8(X, ci, sOff, gr.n_u, sPref, nrb, c0 + 8 * j, c1, v);
                    const float f1 = sF1[side][c], f2 = sF2[side][c];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] *= f1;
                    if constexpr (NAT) slice_store_nat(base, c, j, f2, v);
                    else slice_store<(SA > SB ? SA : SB)>(base, c, j, f2, v);
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                bool started[NCLS];
#pragma unroll
                for (int k = 0; k < NCLS; ++k) started[k] = !first;
                const uint32_t a0 = smem_u32(bufA), b0 = smem_u32(bufB);
#pragma unroll
                for (int s = 1; s <= SA; ++s)
#pragma unroll
                    for (int t = 1; t <= SB; ++t) {
                        if (s + t > LMAX) continue;
                        const int cls = level_class<NCLS>(s + t);
                        const uint32_t d = tmem + (uint32_t)(cls * kST);
#pragma unroll
                        for (int kk = 0; kk < kKC / 16; ++kk) {
                            mma_bf16(d, sw128_desc(a0 + (s - 1) * kPanel + 32 * kk),
                                     sw128_desc(b0 + (t - 1) * kPanel + 32 * kk), idesc, started[cls] ? 1u : 0u);
                            started[cls] = true;
                        }
                    }
                mma_commit(smem_u32(&sBar[b]));
            }
            pending[b] = true;
            first = false;
        }
        // ---- window done: wait for its MMAs, then fold the class sums into acc ------
        for (int b = 0; b < 2; ++b)
            if (pending[b]) {
                if (tid == 0 && !mbar_wait(smem_u32(&sBar[b]), phase[b], kWaitLimitNs)) sFail = 1;
                phase[b] ^= 1u;
                pending[b] = false;
            }
        __syncthreads();
        if (sFail) break;
        tc_fence_after();
        if (flush_act) {
            const int dRa = sDR[0][m], dWa = sDW[0][m];
            const int bs = share ? 0 : 1;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                float cv[NCLS][8];
                const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * q + 8 * h);
#pragma unroll
                for (int k = 0; k < NCLS; ++k) tmem_load8(ta + (uint32_t)(k * kST), cv[k]);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int n = 32 * q + 8 * h + i;
                    float cc[NCLS];
#pragma unroll
                    for (int k = 0; k < NCLS; ++k) cc[k] = cv[k][i];
                    const long long t = window_value<NCLS>(cc);
                    const int dR = min(dRa + sDR[bs][n], 63), dW = min(dWa + sDW[bs][n], 63);
                    acc[8 * h + i] = (acc[8 * h + i] >> dR) + (t >> dW);
                }
            }
        }
        tc_fence_before();
        __syncthreads();                       // tensor memory free for the next window
    }

    // ---- epilogue: int64 -> FP64, one atomic per element (and its mirror) -------------
    if (!sFail && tables_ok && flush_act) {
        const int bs = share ? 0 : 1;
        const int gm = sGcol[0][m];
        const int Ra = sR[0][m];
        if (gm >= 0 && Ra != kNone) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int n = 32 * q + j;
                const int gn = sGcol[bs][n];
                if (gn < 0 || (diag && m > n)) continue;
                const int Rb = sR[bs][n];
                if (Rb == kNone) continue;
                const double val = i64_scaled_to_double(acc[j], Ra + Rb - U);
                if (val == 0.0) continue;
                atomicAdd(&g.G[(int64_t)gm * g.n_cols + gn], val);
                if (SYM && gm != gn) atomicAdd(&g.G[(int64_t)gn * g.n_cols + gm], val);
            }
        }
    }

    // ---- teardown: after a time-out, give the MMAs in flight one more bounded
    // wait; then release the tensor memory ----------------------------------------
    if (sFail && tid == 0) {
        if (g.status) atomicExch(g.status, kDevTimeout);
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait(smem_u32(&sBar[b]), phase[b], kWaitLimitNs);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

template <int SA, int SB, int LMAX, int NCLS, bool SYM, bool SAME, int KX, bool NAT>
cudaError_t launch_tc(const GramTcArgs& g, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<SA, SB, LMAX, NCLS, SYM, SAME, KX, NAT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gram_tc_kernel<SA, SB, LMAX, NCLS, SYM, SAME, KX, NAT><<<(unsigned)g.n_items, kThreads, kSmemDyn, s>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_tc(const GramTcArgs& g, GramMode mode, cudaStream_t s) {
    if (g.n_items == 0) return cudaSuccess;
    // P^T P: 5 fixed-grid slices, levels <= 6, four level classes, windows of
    // 192 rows; P^T Y: 3 slices (the lower two natural bf16), levels <= 4, two
    // classes, windows of 256 rows.  The symmetric modes take the tiles
    // mi <= ni only and mirror them.
    switch (mode) {
        case GramMode::PtP: return launch_tc<5, 5, 6, 4, true, true, 192, false>(g, s);
        case GramMode::PtYSym: return launch_tc<3, 3, 4, 2, true, false, 256, true>(g, s);
        default: return launch_tc<3, 3, 4, 2, false, false, 256, true>(g, s);
    }
}

int gram_tc_tile() { return kST; }
int gram_tc_split_rows() { return 1024; }

}  // namespace femf
