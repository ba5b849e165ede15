// Gram products of FP32 multivectors on the tcgen05 tensor cores with an
// error-free split (C = A^T B over stored blocks, Alg. 8; FP64-accurate
// result).
//
// Numerics.  Work items are runs of at most 192 (P^T P) or 256 (P^T Y) rows
// of a group of consecutive row blocks.  In an item every FP32 value x of union column m
// is normalised by the item's power-of-two bound 2^E_m (|x| < 2^E_m) and
// written as a sum of bf16 slices y_s (every slice exact in bf16, every slice
// product exact in FP32):
//   P^T P  five slices on fixed grids, y_s = q_s 2^(-8 s), |q_1| <= 256,
//          |q_s| <= 128 for s >= 2; products with s + t <= 6 are kept (four
//          slices, s + t <= 5, were measured at 2e-9, above the tolerance);
//   P^T Y  y_1 = q_1 2^-8 on the fixed grid, y_2, y_3 the bf16 roundings of
//          the remainders ("natural" slices); products with s + t <= 4.
// The product of slices s and t has level L = s + t.  The tensor cores sum
// each level class of an item in an FP32 accumulator in tensor memory:
//   P^T P  levels 2, 3 and 4 each on its own: their sums are integers (units
//          2^-16, 2^-24, 2^-32) below 2^24 over 192 rows (level 4: at most
//          (2^15 + 2^14 + 2^15) 192 < 2^24), hence exact whatever the rounding
//          of the tensor-core adder; levels 5 and 6, below 2^-23 of the
//          bound products per row, in a fourth class whose FP32 rounding is
//          immaterial;
//   P^T Y  level 2 exact (its sum is at most 2^16 256 = 2^24 units of 2^-16
//          over 256 rows), levels 3 and 4 together.
// The epilogue turns the class sums of an output element into one integer in
// units of 2^-(8 LMAX) of 2^(E_m + E_n), converts it to FP64 with integer
// operations only (the FP64 pipe of this GPU is slow) and adds it into the
// dense FP64 result with one atomic (symmetric products: into the upper
// triangle, mirrored by a small kernel at the end).
//
// Tiles.  An item computes a 128 x N tile (mi, ni) of its group's union
// columns: operand A of the MMA is the panel of the tile's 128 A columns
// (M = 128 rows of the MMA, one per union column; K = rows of the
// multivector), operand B the panel of its N <= 128 B columns, and
// D[m][n] = sum_k A[m][k] B[n][k] lands in tensor-memory lane m, column n
// (+ 128 per level class).  Panels are staged 64 rows at a time as bf16
// slices in the K-major layout with the 128-byte swizzle (an operand row is
// 64 bf16 = 128 bytes).
//
// Pipeline.  A persistent CTA per SM takes items in a fixed stride and runs
// three roles at once, handing over through mbarriers:
//   producers (16 warps) per item: the group's tables, the column bounds and
//                        exponents; then per 64-row chunk: load, normalise,
//                        slice into a free stage of a two-stage ring;
//   MMA issuer (1 lane)  per chunk: waits for the stage, issues the slice
//                        products (tcgen05.mma kind::f16, bf16 -> FP32),
//                        commits them to free the stage; per item: commits
//                        the accumulators to the epilogue;
//   epilogue (8 warps)   per item: reads the accumulators back (tcgen05.ld;
//                        warp w reaches lanes 32 (w % 4) .. + 31 and takes
//                        half of the tile's columns), releases them, and
//                        adds the results into G.
// The tensor memory holds two accumulator sets of 256 columns: P^T Y (two
// classes) always uses one, alternating, so the epilogue of an item overlaps
// the MMAs of the next; so do the P^T P diagonal tiles with N <= 64 (four
// classes of 64 columns); wider P^T P tiles take both.  Every
// mbarrier wait is bounded in time: on a time-out the kernel sets the status
// word, and every role leaves its loop; the MMA issuer waits (bounded) for its
// MMAs in flight before the tensor memory is freed.
#include <cuda_bf16.h>

#include "fe_internal.h"
#include "tc_common.cuh"

namespace femf {
namespace {

constexpr int kST = 128;                  // output tile edge in union columns (M of the MMA, N <= kST)
constexpr int kKC = 64;                   // rows of a staged chunk: 64 bf16 = one 128-byte swizzle row
// rows of a work item: the level classes summed exactly stay below 2^24
constexpr int kItemRowsPP = 192;          // P^T P (level 4: (2^15 + 2^14 + 2^15) 192 < 2^24)
constexpr int kItemRowsPY = 256;          // P^T Y (level 2: 2^16 256 = 2^24)
constexpr int kPanel = kST * 128;         // bytes of one slice panel (128 operand rows of 128 bytes)
constexpr int kStage = 96 * 1024;         // bytes of one ring stage (both operands of a chunk)
// Warp roles: PW producer warps (groups of 8), 24 - PW epilogue warps, the MMA
// warp last (warp 24).  P^T Y, whose staging is the heavier side, takes 16
// producer warps; P^T P, whose epilogue (four classes) is, takes 16 epilogue
// warps.
constexpr int kMmaWarp = 24;
constexpr int kThreads = 32 * (kMmaWarp + 1);            // 800
constexpr int kBarProd = 1, kBarEpi = 2, kBarProd1 = 3;  // named barriers: producer groups 0 and 1, epilogue
constexpr int kNone = -30000;             // exponent of an all-zero column
constexpr int kMaxRows = (2 * kMaxP + 1) * (2 * kMaxP + 1) * (2 * kMaxP + 1);   // rows of a row block
constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;   // bounded mbarrier waits (0.2 s)

// Tensor-memory loads: thread i of a warp receives lane (32 (warp % 4) + i)
// of the columns loaded.
// The NCLS level classes of 8 consecutive columns: NCLS loads of 32 lanes x 8
// columns (column col + k cstride for class k), then one wait.  The wait (and an
// empty statement for the second half of the registers) is tied to the
// destination registers so that no use moves above it.
template <int NCLS>
__device__ __forceinline__ void tmem_load_classes(uint32_t taddr, uint32_t cstride, float (&v)[NCLS][8]) {
    static_assert(NCLS == 2 || NCLS == 4, "two or four level classes");
    uint32_t r[NCLS][8];
#pragma unroll
    for (int k = 0; k < NCLS; ++k)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[k][0]), "=r"(r[k][1]), "=r"(r[k][2]), "=r"(r[k][3]), "=r"(r[k][4]), "=r"(r[k][5]),
                       "=r"(r[k][6]), "=r"(r[k][7])
                     : "r"(taddr + (uint32_t)k * cstride));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[0][4]), "+r"(r[0][5]),
                   "+r"(r[0][6]), "+r"(r[0][7]), "+r"(r[1][0]), "+r"(r[1][1]), "+r"(r[1][2]), "+r"(r[1][3]),
                   "+r"(r[1][4]), "+r"(r[1][5]), "+r"(r[1][6]), "+r"(r[1][7])
                 :: "memory");
    if constexpr (NCLS == 4)
        asm volatile(""
                     : "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]), "+r"(r[2][4]), "+r"(r[2][5]),
                       "+r"(r[2][6]), "+r"(r[2][7]), "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]),
                       "+r"(r[3][4]), "+r"(r[3][5]), "+r"(r[3][6]), "+r"(r[3][7])
                     :: "memory");
#pragma unroll
    for (int k = 0; k < NCLS; ++k)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[k][i] = __uint_as_float(r[k][i]);
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
// zero) of one 16-byte quad of a union block (slot u, block columns a0 ..
// a0 + 3; consecutive rows of a row block are ld elements apart) as float4.
template <int R>
__device__ __forceinline__ void loadq(const float* __restrict__ X, int u, int a0, int ld, const int64_t* sOff,
                                      int n_u, const int* sPref, int nrb, int kstart, int kend, float4 (&v)[R]) {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kstart >= kend) return;
    int r = 0;
    while (r < nrb - 1 && kstart >= sPref[r + 1]) ++r;
    int e = sPref[r + 1];
    int64_t o = sOff[r * n_u + u];
    int64_t idx = o + (int64_t)(kstart - sPref[r]) * ld + a0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int k = kstart + i;
        if (k < kend) {
            if (k == e) {                     // first row of the next row block (k < kend <= sPref[nrb])
                ++r;
                e = sPref[r + 1];
                o = sOff[r * n_u + u];
                idx = o + a0;
            }
            if (o >= 0) v[i] = __ldg(reinterpret_cast<const float4*>(X + idx));
            idx += ld;
        }
    }
}

// Sources of rows kstart .. kstart+R-1 of one quad (as loadq): nullptr for
// rows at or past kend and for absent blocks (read as zero).
template <int R>
__device__ __forceinline__ void quad_row_srcs(const float* __restrict__ X, int u, int a0, int ld, const int64_t* sOff,
                                              int n_u, const int* sPref, int nrb, int kstart, int kend,
                                              const float* (&src)[R]) {
#pragma unroll
    for (int i = 0; i < R; ++i) src[i] = nullptr;
    if (kstart >= kend) return;
    int r = 0;
    while (r < nrb - 1 && kstart >= sPref[r + 1]) ++r;
    int e = sPref[r + 1];
    int64_t o = sOff[r * n_u + u];
    int64_t idx = o + (int64_t)(kstart - sPref[r]) * ld + a0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int k = kstart + i;
        if (k < kend) {
            if (k == e) {
                ++r;
                e = sPref[r + 1];
                o = sOff[r * n_u + u];
                idx = o + a0;
            }
            if (o >= 0) src[i] = X + idx;
            idx += ld;
        }
    }
}

__device__ __forceinline__ void load8q(const float* __restrict__ X, int u, int a0, int ld, const int64_t* sOff,
                                       int n_u, const int* sPref, int nrb, int kstart, int kend, float4 (&v)[8]) {
    loadq<8>(X, u, a0, ld, sOff, n_u, sPref, nrb, kstart, kend, v);
}

// Component i of a float4
__device__ __forceinline__ float f4c(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// A quad of the tile: the 16-byte chunk (block columns a0 .. a0 + 3) of union
// block u's rows that holds tile columns tc0 .. tc0 + 3; bit i of mask is set
// when block column a0 + i is tile column tc0 + i (not row padding, not
// outside the tile)
struct Quad {
    int u, a0, ld, mask, tc0;
};
__device__ __forceinline__ int quad_pack(int u, int a0, int ld, int mask, int tc0) {
    return u | (a0 << 6) | (ld << 11) | (mask << 19) | ((tc0 + 4) << 23);
}
__device__ __forceinline__ Quad quad_unpack(int q) {
    return Quad{q & 63, (q >> 6) & 31, (q >> 11) & 255, (q >> 19) & 15, ((q >> 23) & 255) - 4};
}

// Rounding to a fixed grid with two additions: for |r| < 2^(k-1), (r + C) - C
// with C = 1.5 2^(k+23) is r rounded to the nearest multiple of 2^k, ties to
// even, as rint(r 2^-k) 2^k (the sum stays in C's binade, whose unit in the
// last place is 2^k, and the difference is exact).  __fadd_rn / __fsub_rn
// keep the compiler from contracting or reassociating the pair.
__device__ __forceinline__ float grid_c(int k) { return __int_as_float(((127 + k + 23) << 23) | 0x400000); }
__device__ __forceinline__ float round_to_grid(float r, float c) { return __fsub_rn(__fadd_rn(r, c), c); }
// Two floats with at most 8 significant bits (exact in bf16) as a bf16 pair,
// a in the low half: their upper 16 bits.
__device__ __forceinline__ uint32_t bf16_pair_exact(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// Slices 8 values (already multiplied by f1) of operand row c into S bf16
// slices y_s = q_s 2^(-8 s) on fixed grids, one 16-byte chunk per slice panel:
// y_s is the residual rounded to the grid 2^(-8 s), the residual loses it
// (exactly), and |q_s| <= 2^8 makes y_s exact in bf16.
// R = 8 values fill the 16-byte chunk j of the row; R = 4 values the half
// h & 1 of chunk h >> 1 (j = h).
template <int S, int R = 8>
__device__ __forceinline__ void slice_store(unsigned char* base, int c, int j, float f2, const float (&v)[R]) {
    static_assert(R == 8 || R == 4, "a 16-byte chunk or half of one");
    float r[R];
#pragma unroll
    for (int i = 0; i < R; ++i) r[i] = v[i] * f2;
    const uint32_t off = R == 8 ? sw_off(c, j) : sw_off(c, j >> 1) + 8u * (uint32_t)(j & 1);
#pragma unroll
    for (int s = 1; s <= S; ++s) {
        const float cs = grid_c(-8 * s);
        uint32_t w[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            const float y0 = round_to_grid(r[2 * i], cs), y1 = round_to_grid(r[2 * i + 1], cs);
            r[2 * i] = __fsub_rn(r[2 * i], y0);
            r[2 * i + 1] = __fsub_rn(r[2 * i + 1], y1);
            w[i] = bf16_pair_exact(y0, y1);
        }
        if constexpr (R == 8)
            *reinterpret_cast<uint4*>(base + (s - 1) * kPanel + off) = make_uint4(w[0], w[1], w[2], w[3]);
        else
            *reinterpret_cast<uint2*>(base + (s - 1) * kPanel + off) = make_uint2(w[0], w[1]);
    }
}

// Three slices with only the first on a fixed grid: y1 = q 2^-8 (|q| <= 256),
// y2 = bf16(x - y1), y3 = bf16(x - y1 - y2).
__device__ __forceinline__ void slice_store_nat(unsigned char* base, int c, int j, float f2, const float (&v)[8]) {
    const uint32_t off = sw_off(c, j);
    const float c1 = grid_c(-8);
    uint32_t w1[4], w2[4], w3[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float r0 = v[2 * i] * f2, r1 = v[2 * i + 1] * f2;
        const float y0 = round_to_grid(r0, c1), y1 = round_to_grid(r1, c1);
        r0 = __fsub_rn(r0, y0);
        r1 = __fsub_rn(r1, y1);
        w1[i] = bf16_pair_exact(y0, y1);
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0, r1);
        r0 -= __low2float(b2);
        r1 -= __high2float(b2);
        const __nv_bfloat162 b3 = __floats2bfloat162_rn(r0, r1);
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

// The item value of one output element from its class sums, as an integer
// in units of 2^-U (U = 8 LMAX) of 2^(E_m + E_n)
template <int NCLS, int U>
__device__ __forceinline__ long long window_value(const float (&c)[NCLS]) {
    if constexpr (NCLS == 4) {   // P^T P: levels 2, 3, 4 exact integers, the rest small
        const int i2 = __float2int_rn(c[0] * pow2f(16));
        const int i3 = __float2int_rn(c[1] * pow2f(24));
        const int i4 = __float2int_rn(c[2] * pow2f(32));
        return ((long long)i2 << (U - 16)) + ((long long)i3 << (U - 24)) + ((long long)i4 << (U - 32)) +
               round_scaled_i64<U, U - 16>(c[3]);
    } else {                     // P^T Y: level 2 exact, the rest
        const int i2 = __float2int_rn(c[0] * pow2f(16));
        return ((long long)i2 << (U - 16)) + round_scaled_i64<U, U - 16>(c[1]);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// named barrier of one warp group (all of its warps converged)
__device__ __forceinline__ void group_sync(int id, int nthreads) {
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Item geometry shared by the three roles
struct ItemGeo {
    bool ok;          // the work-list check passed
    int mi, ni, nrb;
    int wa, wb, N;    // A columns, B columns, MMA N
    bool diag, share;
    int nchunks;
};
template <bool SYM, bool SAME, int ROWS>
__device__ __forceinline__ ItemGeo item_geo(const GramTcItem& it, const GramTcGroup& gr) {
    ItemGeo g;
    g.mi = it.tile & 0xffff;
    g.ni = it.tile >> 16;
    g.nrb = gr.r1 - gr.r0;
    // work-list check: a group has 1..kMaxGroup row blocks of at most kMaxRows
    // rows and 1..kMaxUnion union column blocks (the shared tables depend on
    // it), an item at most ROWS rows
    g.ok = g.nrb >= 1 && g.nrb <= kMaxGroup && gr.n_u >= 1 && gr.n_u <= kMaxUnion && gr.width >= 1 &&
           gr.width <= kMaxUnion * kMaxW && gr.k_rows <= kMaxGroup * kMaxRows && g.mi * kST < gr.width &&
           g.ni * kST < gr.width && !(SYM && g.mi > g.ni) && it.k0 >= 0 && it.k1 <= gr.k_rows && it.k0 < it.k1 &&
           it.k1 - it.k0 <= ROWS && (!SAME || g.mi == g.ni);
    g.wa = min(kST, gr.width - g.mi * kST);
    g.wb = min(kST, gr.width - g.ni * kST);
    g.N = (g.wb + 15) & ~15;
    g.diag = SYM && g.mi == g.ni;
    g.share = SAME;
    g.nchunks = (it.k1 - it.k0 + kKC - 1) / kKC;
    return g;
}

// Metadata of an item that the epilogue needs: global column ids and the
// item exponents of the tile's A and B columns
struct ItemMeta {
    int gcol[2][kST];
    int E[2][kST];
};

// Tensor-memory accumulators: two halves of 256 columns.  An item whose NCLS
// level classes of cs columns each fit in a half (cs = 64 for P^T P diagonal
// tiles with N <= 64, otherwise 128) takes one half, the halves alternating,
// so its MMAs overlap the epilogue of the item before; a wider item takes
// both.  The MMA issuer and the epilogue walk the items in the same order and
// keep the same per-half use counts, which give the mbarrier phases.
struct AccState {
    int hnext;
    int uses[2];
};
struct AccPlan {
    int h0, nh, cs;       // halves h0 .. h0 + nh - 1, class stride in columns
    uint32_t base;        // first tensor-memory column
};
template <int NCLS, bool HALF>
__device__ __forceinline__ AccPlan acc_plan(AccState& st, int N) {
    AccPlan p;
    p.cs = (HALF && N <= kST / 2) ? kST / 2 : kST;
    if (NCLS * p.cs <= 256) {
        p.h0 = st.hnext;
        p.nh = 1;
        st.hnext ^= 1;
    } else {
        p.h0 = 0;
        p.nh = 2;
        st.hnext = 0;
    }
    p.base = 256u * (uint32_t)p.h0;
    return p;
}

// Tables of one item for a group of 256 producer threads (8 warps): the
// group's row-block offsets and row prefix, the tile's columns and their
// 16-byte quads, and the normalisation factors of the columns.
struct ItemTables {
    int64_t off[kMaxGroup * kMaxUnion];   // element offset of block (row block, union slot) or -1
    int pref[kMaxGroup + 1];              // row prefix of the group's row blocks
    int col[2][kST];                      // col_info of tile column c (A side, B side), -1 beyond the tile
    int quad[2][kST];                     // quads (quad_pack), numbered per side
    int nq[2];
    int wcnt[8];
    float f1[2][kST], f2[2][kST];         // x 2^-E = (x f1) f2
};
constexpr int kGroupThreads = 256;

// Builds the offsets, row prefix, tile columns and quads of an item: called
// by the 256 threads of a group (gt = 0..255) with their named barrier.
__device__ __forceinline__ void build_item_tables(ItemTables& T, const GramTcArgs& g, const GramTcItem& it,
                                                  const GramTcGroup& gr, const ItemGeo& ig, int gt, int bar) {
    const int gw = gt >> 5, lane = gt & 31;
    for (int e = gt; e < ig.nrb * gr.n_u; e += kGroupThreads) T.off[e] = g.union_off[gr.u_base + e];
    if (gw == 0) {                                    // row prefix of the group: a warp scan
        int v = lane < ig.nrb ? g.rows[gr.r0 + lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 0) T.pref[0] = 0;
        if (lane < ig.nrb) T.pref[lane + 1] = v;
    }
    // tile columns: A columns on threads 0..127, B columns on 128..255
    const int side_t = gt >> 7, c_t = gt & (kST - 1);
    const int wc_t = side_t ? ig.wb : ig.wa;
    const int ci_t = c_t < wc_t ? g.col_info[gr.c_base + (side_t ? ig.ni : ig.mi) * kST + c_t] : -1;
    T.col[side_t][c_t] = ci_t;
    // quads: one per tile column that starts a 16-byte chunk of its block
    // row (or starts the tile), numbered with warp ballots (warps 0-3: A
    // side, 4-7: B side); the mask marks the chunk's columns that are tile
    // columns of that block
    const int a = (ci_t >> 8) & 0xff;
    const bool head = ci_t >= 0 && ((a & 3) == 0 || c_t == 0);
    const unsigned bal = __ballot_sync(0xffffffffu, head);
    if (lane == 0) T.wcnt[gw] = __popc(bal);
    group_sync(bar, kGroupThreads);
    if (head) {
        int pos = __popc(bal & ((1u << lane) - 1));
        for (int w = 4 * side_t; w < gw; ++w) pos += T.wcnt[w];
        const int u = ci_t >> 16, a0 = a & ~3, tc0 = c_t - (a & 3);
        int mask = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int tc = tc0 + i;
            if (tc >= 0 && tc < wc_t && (T.col[side_t][tc] >> 16) == u) mask |= 1 << i;
        }
        T.quad[side_t][pos] = quad_pack(u, a0, ci_t & 0xff, mask, tc0);
    }
    if (c_t == 0) T.nq[side_t] = T.wcnt[4 * side_t] + T.wcnt[4 * side_t + 1] + T.wcnt[4 * side_t + 2] + T.wcnt[4 * side_t + 3];
    group_sync(bar, kGroupThreads);
}

// Item exponents, before the Gram kernel: for every tile column of an item
// the bound 2^E of |x| over the item's rows (E = kNone for an all-zero
// column), A side then B side (SAME: A only, B = A), as int16 at
// item_exp[item][side][c].  One CTA of 256 threads per item; tasks are
// (quad, 8-row group) with 16-byte loads.
template <bool SYM, bool SAME, int ROWS>
__global__ void __launch_bounds__(kGroupThreads) gram_exp_kernel(const GramTcArgs g) {
    __shared__ ItemTables T;
    __shared__ unsigned sMax[2][kST];
    const int gt = threadIdx.x;
    const int64_t item = blockIdx.x;
    const GramTcItem it = g.items[item];
    const GramTcGroup gr = g.groups[it.group];
    const ItemGeo ig = item_geo<SYM, SAME, ROWS>(it, gr);
    int16_t* out = g.item_exp + item * 2 * kST;
    if (!ig.ok) {                                     // reported by the Gram kernel
        out[gt] = (int16_t)kNone;
        return;
    }
    sMax[gt >> 7][gt & (kST - 1)] = 0u;
    build_item_tables(T, g, it, gr, ig, gt, 1);
    const int ngr = (it.k1 - it.k0 + 7) >> 3;
    for (int side = 0; side < (SAME ? 1 : 2); ++side) {
        const float* X = side ? g.B : g.A;
        const int nq = T.nq[side];
        for (int t = gt; t < nq * ngr; t += kGroupThreads) {
            const Quad qd = quad_unpack(T.quad[side][t % nq]);
            float4 v[8];
            load8q(X, qd.u, qd.a0, qd.ld, T.off, gr.n_u, T.pref, ig.nrb, it.k0 + 8 * (t / nq), it.k1, v);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!((qd.mask >> i) & 1)) continue;
                float mx = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) mx = fmaxf(mx, fabsf(f4c(v[k], i)));
                if (mx > 0.f) atomicMax(&sMax[side][qd.tc0 + i], __float_as_uint(mx));
            }
        }
    }
    __syncthreads();
    const int side = gt >> 7, c = gt & (kST - 1);
    const float mx = __uint_as_float(sMax[SAME ? 0 : side][c]);
    out[gt] = (int16_t)(mx > 0.f ? ilogbf(mx) + 1 : kNone);
}

// SAME: P^T P on diagonal tiles, A = B (one panel); SA, SB slices; LMAX the
// highest level kept; NCLS level classes; SYM upper tiles mirrored; NAT the
// natural three-slice split; NST ring stages (2: a chunk in one 96 KB stage;
// 1: the two operands of a P^T P off-diagonal chunk across the whole 192 KB)
template <int SA, int SB, int LMAX, int NCLS, bool SYM, bool SAME, bool NAT, int NST, int ROWS, int PW, bool HALF>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(const GramTcArgs g) {
    static_assert(!NAT || (SA == 3 && SB == 3), "natural slices: three per operand");
    static_assert(PW == 8 || PW == 16, "one or two producer groups");
    constexpr int EW = kMmaWarp - PW;                          // epilogue warps: 8 or 16
    constexpr int kProdThreads = 32 * PW, kEpiThreads = 32 * EW;
    constexpr int kEpiCols = kST / (EW / 4);                   // tile columns of an epilogue warp
    static_assert(NCLS * kST <= 512, "tensor memory: 128 columns per level class");
    constexpr int U = 8 * LMAX;                 // the epilogue works in units of 2^-U
    // staging task: one quad x RT rows.  P^T P diagonal tiles (one panel, five
    // slices) take 4-row tasks, twice as many, so that the group's threads
    // share them more evenly; the others 8-row tasks
    constexpr int RT = (SAME && !NAT) ? 4 : 8;
    constexpr int kTpq = kKC / RT;              // tasks per quad and chunk
    constexpr int bytesA = SA * kPanel, bytesB = SB * kPanel;
    static_assert(NST == 2 ? (SAME ? bytesA : bytesA + bytesB) <= kStage : bytesA + bytesB <= 2 * kStage,
                  "a chunk fits its stage");
    // One-panel tiles leave the last kStage - bytesA bytes of each stage
    // unused by the MMAs.  There the producer keeps the raw FP32 rows of its
    // tasks, fetched with cp.async one round of tasks ahead (round r of a
    // chunk in the tail of stage r % 2, [row][thread] 16-byte slots), so the
    // loads of the next round are in flight while the current one is sliced.
    constexpr bool kRawPipe = SAME && NST == 2 && PW == 8 && kStage - bytesA >= RT * kGroupThreads * 16;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    unsigned char* ring = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
    __shared__ ItemTables sTab[2];                 // one per producer group
    __shared__ ItemMeta sMeta[2];
    __shared__ __align__(8) uint64_t bFull[2], bEmpty[2], bTFull[2], bTEmpty[2], bMFull[2], bMEmpty[2];
    __shared__ uint32_t sTmem;
    __shared__ volatile int sFail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a kernel launched after this one as dependent may start its CTAs as SMs
    // free up (it reads nothing this kernel writes)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bFull[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bEmpty[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bTFull[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bTEmpty[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bMFull[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bMEmpty[b])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sFail = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sTmem;

    if (warp < PW) {
        // ======================= producers =======================================
        // Groups of 8 warps (two, or one).  Each builds its own copy of every
        // item's tables; with two groups the chunks of the ring alternate
        // between them (chunk n is group n % 2's, in stage n % 2), so that one
        // group loads and slices while the other's chunk is in flight.  With a
        // single group or a single stage (NST 1) group 0 takes every chunk.
        // Group 0 also hands the item metadata to the epilogue.
        const int grp = warp >> 3, gt = tid & (kGroupThreads - 1);
        const int bar = grp == 0 ? kBarProd : kBarProd1;
        ItemTables& T = sTab[grp];
        int chunk_no = 0;
        const int side_t = gt >> 7, c_t = gt & (kST - 1);   // this thread's tile column at table set-up
        // the next item's records are fetched while the current one is worked
        // on (the item, then, once it has arrived, its group)
        GramTcItem it_next{};
        GramTcGroup gr_next{};
        bool have_next = false;
        for (int64_t item = blockIdx.x, il = 0; item < g.n_items; item += gridDim.x, ++il) {
            const GramTcItem it = have_next ? it_next : g.items[item];
            const GramTcGroup gr = have_next ? gr_next : g.groups[it.group];
            have_next = item + gridDim.x < g.n_items;
            if (have_next) it_next = g.items[item + gridDim.x];
            const ItemGeo ig = item_geo<SYM, SAME, ROWS>(it, gr);
            if (!ig.ok) {
                if (tid == 0 && g.status) atomicExch(g.status, kDevBadTile);
                if (have_next) gr_next = g.groups[it_next.group];
                continue;
            }
            const int slot = (int)(il & 1);
            const int nsides = SAME ? 1 : 2;
            // this thread's column: item exponent and global id, loaded with the tables
            const int sd = SAME ? 0 : side_t;
            const int E = g.item_exp[item * 2 * kST + sd * kST + c_t];
            const int wc_t = side_t ? ig.wb : ig.wa;
            const int gcol_t = grp == 0 && c_t < wc_t ? g.col_glob[gr.c_base + (side_t ? ig.ni : ig.mi) * kST + c_t] : -1;
            group_sync(bar, kGroupThreads);                  // the previous item's tables are done with
            build_item_tables(T, g, it, gr, ig, gt, bar);
            if (have_next) gr_next = g.groups[it_next.group];
            // ---- normalisation from the item exponents (|x| < 2^E) ----------------
            {
                const int e = E == kNone ? 0 : E;
                T.f1[side_t][c_t] = pow2f(-(e >> 1));
                T.f2[side_t][c_t] = pow2f(-(e - (e >> 1)));
            }
            if (grp == 0) {
                // the metadata slot is free once the epilogue of item il - 2 is done
                if (gt == 0 && !mbar_wait(smem_u32(&bMEmpty[slot]), ((il >> 1) & 1) ^ 1, kWaitLimitNs)) sFail = 1;
                group_sync(bar, kGroupThreads);
                if (sFail) break;
                sMeta[slot].E[side_t][c_t] = E;
                sMeta[slot].gcol[side_t][c_t] = gcol_t;
                group_sync(bar, kGroupThreads);
                if (gt == 0) mbar_arrive(smem_u32(&bMFull[slot]));
            } else {
                group_sync(bar, kGroupThreads);
                if (sFail) break;
            }
            // ---- chunks of 64 rows: load, normalise, slice into a ring stage -------
            for (int j = 0; j < ig.nchunks; ++j, ++chunk_no) {
                constexpr bool kAlt = NST == 2 && PW == 16;   // chunks alternate between the groups
                if ((kAlt ? (chunk_no & 1) : 0) != grp) continue;
                const int stage = NST == 2 ? (chunk_no & 1) : 0;
                const int use = NST == 2 ? (chunk_no >> 1) : chunk_no;
                const int c0 = it.k0 + kKC * j, c1 = min(it.k1, c0 + kKC);
                // raw rows of task t into the tail of stage `buf` (this thread's slots)
                auto raw_fetch = [&](int t, int buf) {
                    const Quad qd = quad_unpack(T.quad[0][t / kTpq]);
                    const float* src[RT];
                    quad_row_srcs<RT>(g.A, qd.u, qd.a0, qd.ld, T.off, gr.n_u, T.pref, ig.nrb, c0 + RT * (t % kTpq),
                                      c1, src);
                    const uint32_t rb = smem_u32(ring + buf * kStage + bytesA) + 16u * (uint32_t)gt;
#pragma unroll
                    for (int i = 0; i < RT; ++i)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                                         rb + (uint32_t)(i * kGroupThreads * 16)),
                                     "l"(src[i] ? src[i] : g.A), "r"(src[i] ? 16 : 0)
                                     : "memory");
                };
                const int nt_raw = kTpq * T.nq[0];
                if constexpr (kRawPipe) {
                    if (gt < nt_raw) raw_fetch(gt, 0);
                    asm volatile("cp.async.commit_group;\n" ::: "memory");
                }
                if (gt == 0 && !mbar_wait(smem_u32(&bEmpty[stage]), (use & 1) ^ 1, kWaitLimitNs)) sFail = 1;
                group_sync(bar, kGroupThreads);
                if (sFail) break;
                unsigned char* bufA = ring + stage * kStage;
                unsigned char* bufB = SAME ? bufA : bufA + bytesA;
                if constexpr (kRawPipe) {
                    for (int t = gt, r = 0; t < nt_raw; t += kGroupThreads, ++r) {
                        if (t + kGroupThreads < nt_raw) raw_fetch(t + kGroupThreads, (r + 1) & 1);
                        asm volatile("cp.async.commit_group;\n" ::: "memory");
                        asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // round r has landed
                        const Quad qd = quad_unpack(T.quad[0][t / kTpq]);
                        const int jj = t % kTpq;
                        const unsigned char* rb = ring + (r & 1) * kStage + bytesA + 16 * gt;
                        float4 v[RT];
#pragma unroll
                        for (int i = 0; i < RT; ++i)
                            v[i] = *reinterpret_cast<const float4*>(rb + i * kGroupThreads * 16);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (!((qd.mask >> i) & 1)) continue;
                            const int tc = qd.tc0 + i;
                            const float f1 = T.f1[0][tc], f2 = T.f2[0][tc];
                            float x[RT];
#pragma unroll
                            for (int k = 0; k < RT; ++k) x[k] = f4c(v[k], i) * f1;
                            slice_store<(SA > SB ? SA : SB), RT>(bufA, tc, jj, f2, x);
                        }
                    }
                    asm volatile("cp.async.wait_all;\n" ::: "memory");
                } else {
                    // operand rows beyond the tile's columns are never read back:
                    // they are left as they are.  Tasks are (quad, RT-row group),
                    // the A side's then the B side's in one range, so that the
                    // group's threads share both sides' tasks evenly.
                    // Neighbouring threads take the row groups of a quad, so
                    // that the slice stores of a warp (16 or 8 bytes each) cover
                    // whole 128-byte swizzled rows (no bank conflicts).
                    const int nt0 = kTpq * T.nq[0], nt = nt0 + (nsides > 1 ? kTpq * T.nq[1] : 0);
                    for (int t = gt; t < nt; t += kGroupThreads) {
                        const int side = t >= nt0 ? 1 : 0;
                        const int ts = t - side * nt0;
                        const float* X = side ? g.B : g.A;
                        unsigned char* base = side ? bufB : bufA;
                        const Quad qd = quad_unpack(T.quad[side][ts / kTpq]);
                        const int jj = ts % kTpq;
                        float4 v[RT];
                        loadq<RT>(X, qd.u, qd.a0, qd.ld, T.off, gr.n_u, T.pref, ig.nrb, c0 + RT * jj, c1, v);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (!((qd.mask >> i) & 1)) continue;
                            const int tc = qd.tc0 + i;
                            const float f1 = T.f1[side][tc], f2 = T.f2[side][tc];
                            float x[RT];
#pragma unroll
                            for (int k = 0; k < RT; ++k) x[k] = f4c(v[k], i) * f1;
                            if constexpr (NAT) slice_store_nat(base, tc, jj, f2, x);
                            else slice_store<(SA > SB ? SA : SB), RT>(base, tc, jj, f2, x);
                        }
                    }
                }
                fence_async_smem();
                group_sync(bar, kGroupThreads);
                if (gt == 0) mbar_arrive(smem_u32(&bFull[stage]));
            }
            if (sFail) break;
        }
    } else if (warp < kMmaWarp) {
        // ======================= epilogue ========================================
        const int ew = warp - PW;                         // 0 .. EW - 1
        const int quad = ew & 3;                          // tensor-memory lanes 32 quad .. + 31
        const int m = 32 * quad + lane;                   // tile row (A column) of this thread
        const int part = ew >> 2;                         // tile columns [kEpiCols part, + kEpiCols)
        const int etid = tid - kProdThreads;
        AccState est{0, {0, 0}};
        for (int64_t item = blockIdx.x, il = 0; item < g.n_items; item += gridDim.x, ++il) {
            const GramTcItem it = g.items[item];
            const GramTcGroup gr = g.groups[it.group];
            const ItemGeo ig = item_geo<SYM, SAME, ROWS>(it, gr);
            if (!ig.ok) continue;
            const int slot = (int)(il & 1);
            const AccPlan ap = acc_plan<NCLS, HALF>(est, ig.N);
            if (etid == 0) {
                for (int h = ap.h0; h < ap.h0 + ap.nh; ++h)
                    if (!mbar_wait(smem_u32(&bTFull[h]), (uint32_t)(est.uses[h] & 1), kWaitLimitNs)) sFail = 1;
                if (!mbar_wait(smem_u32(&bMFull[slot]), (uint32_t)((il >> 1) & 1), kWaitLimitNs)) sFail = 1;
            }
            group_sync(kBarEpi, kEpiThreads);
            if (sFail) break;
            tc_fence_after();
            const ItemMeta& mt = sMeta[slot];
            const int gm = mt.gcol[0][m], Ea = mt.E[0][m];
            const uint32_t tbase = tmem + ((uint32_t)(32 * quad) << 16) + ap.base;
#pragma unroll 1
            for (int h = 0; h < kEpiCols / 8; ++h) {
                const int n0 = kEpiCols * part + 8 * h;
                // warp-uniform skips: lanes beyond the tile's A columns, columns
                // beyond N, or wholly below the diagonal of a diagonal tile
                if (32 * quad >= ig.wa || n0 >= ig.N || (ig.diag && n0 + 7 < 32 * quad)) continue;
                float cv[NCLS][8];
                tmem_load_classes<NCLS>(tbase + (uint32_t)n0, (uint32_t)ap.cs, cv);
                if (gm < 0 || Ea == kNone) continue;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int n = n0 + i;
                    const int gn = mt.gcol[1][n], Eb = mt.E[1][n];
                    if (gn < 0 || Eb == kNone || (ig.diag && m > n)) continue;
                    float cc[NCLS];
                    bool nz = false;
#pragma unroll
                    for (int k = 0; k < NCLS; ++k) {
                        cc[k] = cv[k][i];
                        nz = nz || cc[k] != 0.f;
                    }
                    if (!nz) continue;                        // columns that share no row of the item
                    const double val = i64_scaled_to_double(window_value<NCLS, U>(cc), Ea + Eb - U);
                    if (val == 0.0) continue;
                    // symmetric products: the upper triangle only (gm <= gn
                    // here, union columns being in ascending global order);
                    // mirror_upper fills the lower one afterwards
                    atomicAdd(&g.G[(int64_t)gm * g.n_cols + gn], val);
                }
            }
            tc_fence_before();
            group_sync(kBarEpi, kEpiThreads);                 // the accumulators and the metadata are read
            if (etid == 0) {
                for (int h = ap.h0; h < ap.h0 + ap.nh; ++h) mbar_arrive(smem_u32(&bTEmpty[h]));
                mbar_arrive(smem_u32(&bMEmpty[slot]));
            }
            for (int h = ap.h0; h < ap.h0 + ap.nh; ++h) ++est.uses[h];
        }
    } else {
        // ======================= MMA issuer (one lane) ===========================
        AccState mst{0, {0, 0}};
        int chunk_no = 0;
        uint32_t last_bar = 0, last_parity = 0;
        bool issued = false;
        for (int64_t item = blockIdx.x, il = 0; item < g.n_items; item += gridDim.x, ++il) {
            const GramTcItem it = g.items[item];
            const GramTcGroup gr = g.groups[it.group];
            const ItemGeo ig = item_geo<SYM, SAME, ROWS>(it, gr);
            if (!ig.ok) continue;
            const AccPlan ap = acc_plan<NCLS, HALF>(mst, ig.N);
            bool fail = false;
            if (lane == 0) {
                for (int h = ap.h0; h < ap.h0 + ap.nh && !fail; ++h)
                    fail = !mbar_wait(smem_u32(&bTEmpty[h]), (uint32_t)((mst.uses[h] & 1) ^ 1), kWaitLimitNs);
                if (!fail) tc_fence_after();
                const uint32_t idesc = bf16_idesc(128, ig.N);
                const uint32_t dset = tmem + ap.base;
                bool started[NCLS];
#pragma unroll
                for (int k = 0; k < NCLS; ++k) started[k] = false;
                for (int j = 0; j < ig.nchunks && !fail; ++j, ++chunk_no) {
                    const int stage = NST == 2 ? (chunk_no & 1) : 0;
                    const int use = NST == 2 ? (chunk_no >> 1) : chunk_no;
                    if (!mbar_wait(smem_u32(&bFull[stage]), (uint32_t)(use & 1), kWaitLimitNs)) {
                        fail = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(ring + stage * kStage);
                    const uint32_t b0 = SAME ? a0 : a0 + bytesA;
#pragma unroll
                    for (int s = 1; s <= SA; ++s)
#pragma unroll
                        for (int t = 1; t <= SB; ++t) {
                            if (s + t > LMAX) continue;
                            const int cls = level_class<NCLS>(s + t);
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; ++kk) {
                                // the first product of each class in the item starts its sum
                                mma_bf16(dset + (uint32_t)(cls * ap.cs), sw128_desc(a0 + (s - 1) * kPanel + 32 * kk),
                                         sw128_desc(b0 + (t - 1) * kPanel + 32 * kk), idesc, started[cls] ? 1u : 0u);
                                started[cls] = true;
                            }
                        }
                    mma_commit(smem_u32(&bEmpty[stage]));
                    last_bar = smem_u32(&bEmpty[stage]);
                    last_parity = (uint32_t)(use & 1);
                    issued = true;
                }
                if (!fail) {
                    for (int h = ap.h0; h < ap.h0 + ap.nh; ++h) {
                        mma_commit(smem_u32(&bTFull[h]));
                        last_bar = smem_u32(&bTFull[h]);
                        last_parity = (uint32_t)(mst.uses[h] & 1);
                    }
                }
                if (fail) sFail = 1;
            }
            for (int h = ap.h0; h < ap.h0 + ap.nh; ++h) ++mst.uses[h];
            __syncwarp();
            if (sFail) break;
        }
        // after a failure, let the MMAs in flight finish before the tensor
        // memory is freed
        if (lane == 0 && sFail && issued) mbar_wait(last_bar, last_parity, kWaitLimitNs);
        __syncwarp();
    }

    if (sFail && tid == 0 && g.status) atomicExch(g.status, kDevTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// G[n][m] = G[m][n] for m < n: the lower triangle of a symmetric product
// from the upper one that the Gram kernel accumulated.
__global__ void __launch_bounds__(256) mirror_upper_kernel(double* __restrict__ G, int n) {
    const int64_t total = (int64_t)n * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / n), c = (int)(idx - (int64_t)r * n);
        if (r > c) G[idx] = G[(int64_t)c * n + r];
    }
}

cudaError_t mirror_upper(double* G, int n, cudaStream_t s) {
    const int64_t total = (int64_t)n * n;
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    mirror_upper_kernel<<<grid, 256, 0, s>>>(G, n);
    return cudaGetLastError();
}

// The item exponents of g's items: one CTA per item.
template <bool SYM, bool SAME, int ROWS>
cudaError_t launch_exp(const GramTcArgs& g, cudaStream_t s) {
    if (g.n_items == 0) return cudaSuccess;
    gram_exp_kernel<SYM, SAME, ROWS><<<(unsigned)g.n_items, kGroupThreads, 0, s>>>(g);
    return cudaGetLastError();
}

// The persistent Gram kernel over g's items (their exponents computed before).
// dependent: launched with programmatic stream serialisation, so that its
// CTAs take the SMs that the previous kernel's CTAs leave while the rest of
// that kernel still runs (the previous kernel triggers at its start).  Only
// for a kernel that reads nothing the previous one writes.
template <int SA, int SB, int LMAX, int NCLS, bool SYM, bool SAME, bool NAT, int NST, int ROWS, int PW, bool HALF>
cudaError_t launch_tc(const GramTcArgs& g, cudaStream_t s, bool dependent = false) {
    constexpr int smem = 2 * kStage + 1024;
    auto kern = gram_tc_kernel<SA, SB, LMAX, NCLS, SYM, SAME, NAT, NST, ROWS, PW, HALF>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (g.n_items == 0) return cudaSuccess;
    const int sms = usable_sms(g.sm_limit);
    if (sms < 1) return cudaErrorInvalidDevice;
    const unsigned grid = (unsigned)std::min<int64_t>(g.n_items, (int64_t)sms);
    if (!dependent) {
        kern<<<grid, kThreads, smem, s>>>(g);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g);
}

}  // namespace

cudaError_t launch_gram_tc(const GramTcArgs& g, GramMode mode, cudaStream_t s) {
    // P^T P: 5 fixed-grid slices, levels <= 6, four level classes; the
    // diagonal tiles (listed first, n_items_diag of them) stage one panel,
    // the off-diagonal ones (groups wider than 128 columns) two panels in a
    // single 192 KB stage.  P^T Y: 3 slices (the lower two natural bf16),
    // levels <= 4, two classes.  The symmetric modes take the tiles
    // mi <= ni only and mirror them.
    switch (mode) {
        case GramMode::PtP: {
            GramTcArgs d = g, o = g;
            d.n_items = g.n_items_diag;
            o.items = g.items + g.n_items_diag;
            o.item_exp = g.item_exp + g.n_items_diag * 2 * kST;
            o.n_items = g.n_items - g.n_items_diag;
            // both exponent passes first; the off-diagonal tiles then fill the
            // SMs that the diagonal kernel's CTAs leave as they finish
            cudaError_t e = launch_exp<true, true, kItemRowsPP>(d, s);
            if (e == cudaSuccess) e = launch_exp<true, false, kItemRowsPP>(o, s);
            if (e == cudaSuccess) e = launch_tc<5, 5, 6, 4, true, true, false, 2, kItemRowsPP, 8, true>(d, s);
            if (e == cudaSuccess)
                e = launch_tc<5, 5, 6, 4, true, false, false, 1, kItemRowsPP, 8, false>(o, s, d.n_items > 0);
            if (e == cudaSuccess) e = mirror_upper(g.G, g.n_cols, s);
            return e;
        }
        case GramMode::PtYSym: {
            cudaError_t e = launch_exp<true, false, kItemRowsPY>(g, s);
            if (e == cudaSuccess) e = launch_tc<3, 3, 4, 2, true, false, true, 2, kItemRowsPY, 16, false>(g, s);
            if (e == cudaSuccess) e = mirror_upper(g.G, g.n_cols, s);
            return e;
        }
        default: {
            cudaError_t e = launch_exp<false, false, kItemRowsPY>(g, s);
            if (e == cudaSuccess) e = launch_tc<3, 3, 4, 2, false, false, true, 2, kItemRowsPY, 16, false>(g, s);
            return e;
        }
    }
}

int gram_tc_tile() { return kST; }
int gram_tc_item_rows(bool pp) { return pp ? kItemRowsPP : kItemRowsPY; }

}  // namespace femf
