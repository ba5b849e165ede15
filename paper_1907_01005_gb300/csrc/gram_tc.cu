// Gram products of FP32 multivectors on the tensor cores with an error-free
// split (C = A^T B over stored blocks, Alg. 8; FP64-accurate accumulation).
//
// Rows are processed in windows of KW rows.  In a window every FP32 value x
// of union column m is normalised by the window's own power-of-two bound
// 2^E (|x| < 2^E, E per column and window) and written as a sum of slices
//   x 2^-E = sum_s y_s ,  y_s = q_s 2^(-8 s),  q_s integer, |q_s| <= 256,
// so every y_s is exact in bf16 and every slice product is exact in FP32.
// The product of slices s and t belongs to level L = s + t (weight
// 2^(-8 L)); levels above LMAX are dropped.  Per window the tensor cores
// (mma.sync m16n8k16, bf16 -> FP32) sum
//   level 2 and level 3 in accumulators of their own: their window sums are
//     integers (in units of 2^-16, 2^-24) below 2^23, hence exact whatever
//     the rounding of the tensor-core adder;
//   levels 4..LMAX together in a third accumulator: their weight is below
//     2^-32 of the result, so the FP32 rounding there is immaterial.
// After each window the three sums are converted to integers in units of
// 2^-(8 LMAX) and combined into an int64 per output element, scaled by
// 2^(E_m(w) + E_n(w)) relative to a running per-column reference exponent
// R (the largest window exponent seen so far): the accumulator is shifted
// right when R grows and the window value when it is below R.  The dropped
// bits are below 2^-(8 LMAX) of the reference scale per window.
//
// The error is set by the residual after the last slice (2^(-8S-1) of the
// column bound) and by the first dropped level: P^T Y uses 3 slices and
// levels <= 4 (6 products, ~2^-25), P^T P 5 slices and levels <= 6
// (15 products, ~2^-40).  The int64 is converted to FP64 with integer
// operations only (the FP64 pipe of this GPU runs at 1/64 of the FP32
// rate) and added into the dense FP64 result with one atomic per element.
//
// Work item: (group of consecutive row blocks, 64 x 64 super-tile of the
// group's union columns, range of the group's rows).  8 warps, each owning
// a 16 x 32 sub-tile (four m16n8k16 tiles); slices are staged in shared
// memory as [column][row] bf16 rows with XOR-swizzled 16-byte chunks and
// read with ldmatrix.
#include <cuda_bf16.h>

#include "fe_internal.h"

namespace femf {
namespace {

constexpr int kST = 64;          // super-tile edge (union columns)
constexpr int kThreads = 256;    // 8 warps: 4 (m16) x 2 (n32)
constexpr int kNone = -30000;    // exponent of an all-zero column
constexpr int kMaxRows = (2 * kMaxP + 1) * (2 * kMaxP + 1) * (2 * kMaxP + 1);   // rows of a row block

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

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

// Shared-memory byte offset of (column c, 16-byte chunk kc) in a slice of
// kST columns x KW rows.  The low 3 bits of the chunk index are XOR-ed with
// the column's low 3 bits (ldmatrix reads 8 consecutive columns at one
// chunk) and with bit 3 of the chunk index moved to bit 1 (a staging store
// phase writes 2 columns x 4 row segments, whose chunks differ in bits 2
// and 3): both patterns hit 8 different 16-byte bank groups.
// With NSEG = 8 row segments of two chunks, bit 3 of the chunk index goes to
// bit 0 instead: the 8 segments of one column, which store together, then
// also hit 8 different bank groups.
template <int KW, int NSEG = 4>
__device__ __forceinline__ unsigned chunk_off(int c, int kc) {
    if constexpr (NSEG == 8) return (unsigned)(c * (KW * 2) + ((kc ^ (c & 7) ^ ((kc >> 3) & 1)) << 4));
    return (unsigned)(c * (KW * 2) + ((kc ^ (c & 7) ^ (((kc >> 3) & 1) << 1)) << 4));
}

// Rounds v 2^U (|v 2^U| < 2^62, v a float) to an int64 with two 32-bit
// conversions (the 64-bit one runs on the FP64 pipe): the high part on the
// 2^-H grid, then the exact remainder.
template <int U, int H>
__device__ __forceinline__ long long round_scaled_i64(float v) {
    const float hi = rintf(v * pow2f(H));
    const float rem = fmaf(-hi, pow2f(-H), v);               // exact
    return ((long long)(int)hi << (U - H)) + (long long)__float2int_rn(rem * pow2f(U));
}

// Loads rows kstart .. kstart+SEG-1 of the group (those at or past kend
// read as zero) of one union column into registers and returns max |x|.
// Consecutive rows of a row block are ld elements apart.  A segment that
// touches at most two row blocks (always for p >= 2, whose row blocks hold
// at least (2p)^3 >= SEG rows) gets its addresses from two bases, so all
// loads are independent; otherwise the rows are walked one by one.
template <int SEG>
__device__ __forceinline__ float load_window(const float* __restrict__ X, int ci, const int64_t* sOff, int n_u,
                                             const int* sPref, int nrb, int kstart, int kend, float (&v)[SEG]) {
#pragma unroll
    for (int i = 0; i < SEG; ++i) v[i] = 0.f;
    if (ci < 0 || kstart >= kend) return 0.f;
    const int slot = ci >> 16, a = (ci >> 8) & 0xff, ld = ci & 0xff;
    int r = 0;
    while (r < nrb - 1 && kstart >= sPref[r + 1]) ++r;
    const int end_r = sPref[r + 1];
    float mx = 0.f;
    if (r + 1 >= nrb || sPref[r + 2] >= kstart + SEG) {
        const int64_t o0 = sOff[r * n_u + slot];
        const int64_t o1 = r + 1 < nrb ? sOff[(r + 1) * n_u + slot] : -1;
        const int64_t b0 = o0 + (int64_t)(kstart - sPref[r]) * ld + a;   // row kstart + i -> b0 + i ld
        const int64_t b1 = o1 + a - (int64_t)end_r * ld;                  // row k >= end_r -> b1 + k ld
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
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
        for (int i = 0; i < SEG; ++i) {
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
#pragma unroll
    for (int i = 0; i < SEG; ++i) mx = fmaxf(mx, fabsf(v[i]));
    return mx;
}

// Column exponent of this window and the update of the running reference R
// (kept in a register by each of the column's four staging lanes; the first
// of them publishes the shifts for the flush and R for the epilogue).
struct WinExp {
    int dR, dW;       // accumulator shift (growth of R), window-value shift (R - E)
    float f1, f2;     // x 2^-E = (x * f1) * f2 without underflow
};
__device__ __forceinline__ WinExp window_exponent(float mx, int& R) {
    const int E = mx > 0.f ? ilogbf(mx) + 1 : kNone;
    const int newR = E > R ? E : R;
    WinExp w;
    w.dR = (R == kNone) ? 0 : min(newR - R, 63);
    w.dW = (E == kNone) ? 63 : min(newR - E, 63);
    R = newR;
    const int e = (E == kNone) ? 0 : E;
    w.f1 = pow2f(-(e >> 1));
    w.f2 = pow2f(-(e - (e >> 1)));
    return w;
}

// Slices a thread's SEG values (column c, rows seg*SEG ..) into S bf16
// slices y_s = q_s 2^(-8 s) and stores them as SEG/8 16-byte chunks each.
template <int S, int SEG, int KW, int NSEG = 4>
__device__ __forceinline__ void slice_store(unsigned char* base, int c, int seg, float f1, float f2,
                                            const float (&v)[SEG]) {
    constexpr int SLICE = kST * KW * 2;
#pragma unroll
    for (int ch = 0; ch < SEG / 8; ++ch) {
        float r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = (v[ch * 8 + i] * f1) * f2;
        const unsigned off = chunk_off<KW, NSEG>(c, seg * (SEG / 8) + ch);
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
            *reinterpret_cast<uint4*>(base + (s - 1) * SLICE + off) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Three slices with only the first on a fixed grid: y1 = q 2^-8 (|q| <= 256),
// y2 = bf16(x - y1), y3 = bf16(x - y1 - y2).  Products y1 y1' stay on the
// 2^-16 grid (exact window sums); the others are exact FP32 numbers whose
// window sums are rounded, at a weight of 2^-8 of the result or less.
template <int SEG, int KW, int NSEG = 4>
__device__ __forceinline__ void slice_store_nat(unsigned char* base, int c, int seg, float f1, float f2,
                                                const float (&v)[SEG]) {
    constexpr int SLICE = kST * KW * 2;
#pragma unroll
    for (int ch = 0; ch < SEG / 8; ++ch) {
        const unsigned off = chunk_off<KW, NSEG>(c, seg * (SEG / 8) + ch);
        uint32_t w1[4], w2[4], w3[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float r0 = (v[ch * 8 + 2 * i] * f1) * f2, r1 = (v[ch * 8 + 2 * i + 1] * f1) * f2;
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
        *reinterpret_cast<uint4*>(base + SLICE + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        *reinterpret_cast<uint4*>(base + 2 * SLICE + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
    }
}

template <int SA, int SB, int LMAX, bool SYM, bool SAME, int KW, bool NAT>
__global__ void __launch_bounds__(kThreads, 2) gram_tc_kernel(const GramTcArgs g) {
    static_assert(KW % 32 == 0 && KW <= 128, "window rows");
    static_assert(!NAT || (SA == 3 && SB == 3), "natural slices: three per operand");
    // staging: NSEG lanes per column, SEG rows each; 128-row windows take
    // two passes of 32 columns (16 rows a lane keeps the registers in bounds)
    constexpr int NSEG = KW >= 128 ? 8 : 4;
    constexpr int SEG = KW / NSEG;                // rows per staging thread
    constexpr int CPP = kThreads / NSEG;          // columns per pass
    constexpr int NPASS = kST / CPP;
    constexpr int SLICE = kST * KW * 2;           // bytes per staged slice
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* As = smem;
    unsigned char* Bs = smem + SA * SLICE;
    __shared__ int64_t sOff[kMaxGroup * kMaxUnion];
    __shared__ int sColA[kST], sColB[kST], sGcolA[kST], sGcolB[kST];
    __shared__ int sPref[kMaxGroup + 1];
    __shared__ int sR[2][kST], sDR[2][kST], sDW[2][kST];

    const GramTcItem it = g.items[blockIdx.x];
    const GramTcGroup gr = g.groups[it.group];
    const int mi = it.tile & 0xffff, ni = it.tile >> 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrb = gr.r1 - gr.r0;
    // Work-list check: a group has 1..kMaxGroup row blocks of at most kMaxRows
    // rows and at most kMaxUnion union column blocks (the shared tables and
    // the int64 bound depend on it); a malformed item sets the status word
    // and leaves G untouched.
    if (nrb < 1 || nrb > kMaxGroup || gr.n_u < 1 || gr.n_u > kMaxUnion || gr.width < 1 ||
        gr.width > kMaxUnion * kMaxW || gr.k_rows > kMaxGroup * kMaxRows || mi * kST >= gr.width ||
        ni * kST >= gr.width || it.k0 < 0 || it.k1 > gr.k_rows || it.k0 >= it.k1) {
        if (tid == 0 && g.status) atomicExch(g.status, kDevBadTile);
        return;
    }
    const bool diag = SYM && mi == ni;            // diagonal super-tile of a symmetric product
    const bool share = SAME && mi == ni;          // ... whose B columns are A's own (B = A)

    // ---- group tables ------------------------------------------------------
    for (int e = tid; e < nrb * gr.n_u; e += kThreads) sOff[e] = g.union_off[gr.u_base + e];
    if (tid < kST) {
        const int ma = mi * kST + tid, nb = ni * kST + tid;
        sColA[tid] = ma < gr.width ? g.col_info[gr.c_base + ma] : -1;
        sGcolA[tid] = ma < gr.width ? g.col_glob[gr.c_base + ma] : -1;
        sColB[tid] = nb < gr.width ? g.col_info[gr.c_base + nb] : -1;
        sGcolB[tid] = nb < gr.width ? g.col_glob[gr.c_base + nb] : -1;
    }
    if (tid == 0) {
        sPref[0] = 0;
        for (int r = 0; r < nrb; ++r) sPref[r + 1] = sPref[r] + g.rows[gr.r0 + r];
    }
    __syncthreads();
    if (sPref[nrb] != gr.k_rows) {                // the row walk relies on it
        if (tid == 0 && g.status) atomicExch(g.status, kDevBadTile);
        return;
    }

    const int bo = share ? 0 : 1;                 // operand index of B's column state
    const int wm = (warp >> 1) * 16, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tig = lane & 3;
    const bool wact = (mi * kST + wm < gr.width) && (ni * kST + wn < gr.width) && (!diag || wm < wn + 32);
    const int seg = tid % NSEG;                   // a column's NSEG row segments sit in one warp
    int RA[NPASS], RB[NPASS];                     // running reference exponents of this thread's columns
#pragma unroll
    for (int ps = 0; ps < NPASS; ++ps) RA[ps] = RB[ps] = kNone;

    long long acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[j][v] = 0;

    const unsigned As_s = (unsigned)__cvta_generic_to_shared(As);
    const unsigned Bs_s = (unsigned)__cvta_generic_to_shared(share ? As : Bs);

    for (int k0 = it.k0; k0 < it.k1; k0 += KW) {
        __syncthreads();                           // tables ready; previous window's MMAs and flush done
        // ---- per operand: load, column bound (NSEG lanes of a column), slices
#pragma unroll
        for (int ps = 0; ps < NPASS; ++ps) {
            const int c = ps * CPP + tid / NSEG;
            {
                const int ca = sColA[c];
                float v[SEG];
                float mx = load_window<SEG>(g.A, ca, sOff, gr.n_u, sPref, nrb, k0 + seg * SEG, it.k1, v);
#pragma unroll
                for (int o = 1; o < NSEG; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                const WinExp e = window_exponent(mx, RA[ps]);
                if (seg == 0) {
                    sDR[0][c] = e.dR;
                    sDW[0][c] = e.dW;
                    sR[0][c] = RA[ps];
                }
                if (ca >= 0) {
                    if constexpr (NAT) slice_store_nat<SEG, KW, NSEG>(As, c, seg, e.f1, e.f2, v);
                    else slice_store<SA, SEG, KW, NSEG>(As, c, seg, e.f1, e.f2, v);
                }
            }
            if (!share) {
                const int cb = sColB[c];
                float v[SEG];
                float mx = load_window<SEG>(g.B, cb, sOff, gr.n_u, sPref, nrb, k0 + seg * SEG, it.k1, v);
#pragma unroll
                for (int o = 1; o < NSEG; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                const WinExp e = window_exponent(mx, RB[ps]);
                if (seg == 0) {
                    sDR[1][c] = e.dR;
                    sDW[1][c] = e.dW;
                    sR[1][c] = RB[ps];
                }
                if (cb >= 0) {
                    if constexpr (NAT) slice_store_nat<SEG, KW, NSEG>(Bs, c, seg, e.f1, e.f2, v);
                    else slice_store<SB, SEG, KW, NSEG>(Bs, c, seg, e.f1, e.f2, v);
                }
            }
        }
        __syncthreads();
        if (!wact) continue;

    // ---- tensor-core products of the window -------------------------------
        float wacc[3][4][4];
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) wacc[l][j][v] = 0.f;
        const int am = wm + (lane & 15);
        const int bn = wn + (lane & 7) + ((lane >> 4) << 3);
#pragma unroll
        for (int ks = 0; ks < KW / 16; ++ks) {
            uint32_t af[SA][4];
#pragma unroll
            for (int s = 0; s < SA; ++s) ldsm_x4(af[s], As_s + s * SLICE + chunk_off<KW, NSEG>(am, 2 * ks + (lane >> 4)));
#pragma unroll
            for (int p = 0; p < 2; ++p) {                 // pairs of n8 tiles
                const unsigned boff = chunk_off<KW, NSEG>(bn + 16 * p, 2 * ks + ((lane >> 3) & 1));
#pragma unroll
                for (int t = 1; t <= SB; ++t) {            // one B slice at a time
                    uint32_t bf[4];
                    ldsm_x4(bf, Bs_s + (t - 1) * SLICE + boff);
#pragma unroll
                    for (int s = 1; s <= SA; ++s) {
                        const int L = s + t;
                        if (L > LMAX) continue;
                        const int cls = L == 2 ? 0 : ((L == 3 && !NAT) ? 1 : 2);
                        mma_bf16(wacc[cls][2 * p], af[s - 1], bf[0], bf[1]);
                        mma_bf16(wacc[cls][2 * p + 1], af[s - 1], bf[2], bf[3]);
                    }
                }
            }
        }
        // ---- flush: exact window value into the int64 accumulators -----------
        // In units of 2^-(8 LMAX) the window value is
        //   t = i2 2^(8 LMAX - 16) + i3 2^(8 LMAX - 24) + hi 2^(4 LMAX) + lo
        // (i2, i3: the exact level-2 / level-3 sums; hi, lo: the levels-4+ sum
        // rounded on the 2^-(4 LMAX) grid and its remainder).  The first three
        // share the factor 2^(4 LMAX) and their sum fits in 32 bits
        // (|i2| <= 2^22 x 2^8, |i3| <= 2^23, |hi| <= 2^16 for P^T P; |i2| <= 2^23,
        // |hi| <= 2^15 for P^T Y), so t is one 32-bit sum shifted, plus lo.
        int dRa[2], dWa[2], dRb[8], dWb[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            dRa[h] = sDR[0][wm + gid + 8 * h];
            dWa[h] = sDW[0][wm + gid + 8 * h];
        }
        int grow = dRa[0] | dRa[1];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int n = wn + 8 * (q >> 1) + 2 * tig + (q & 1);
            dRb[q] = sDR[bo][n];
            dWb[q] = sDW[bo][n];
            grow |= dRb[q];
        }
        // the reference exponents grow in few windows: shift the accumulators
        // only when some lane of the warp needs it
        const bool any_grow = __any_sync(0xffffffffu, grow != 0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int q = 2 * j + (v & 1);
                const int h = v >> 1;
                const float w2 = wacc[2][j][v];
                const float hiF = rintf(w2 * pow2f(4 * LMAX));
                const int lo = __float2int_rn(fmaf(-hiF, pow2f(-4 * LMAX), w2) * pow2f(8 * LMAX));
                int top = (__float2int_rn(wacc[0][j][v] * pow2f(16)) << (4 * LMAX - 16)) + (int)hiF;
                if constexpr (!NAT) top += __float2int_rn(wacc[1][j][v] * pow2f(24)) << (4 * LMAX - 24);
                const long long t = ((long long)top << (4 * LMAX)) + lo;
                const int shW = min(dWa[h] + dWb[q], 63);
                if (any_grow) acc[j][v] >>= min(dRa[h] + dRb[q], 63);
                acc[j][v] += t >> shW;
            }
    }
    if (!wact) return;

    // ---- epilogue: int64 -> FP64, one atomic per element --------------------
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int m = wm + gid + (v >= 2 ? 8 : 0);
            const int n = wn + 8 * j + tig * 2 + (v & 1);
            const int gm = sGcolA[m], gn = sGcolB[n];
            if (gm < 0 || gn < 0) continue;
            if (diag && m > n) continue;                 // lower half of a diagonal tile: mirrored below
            const int Ra = sR[0][m], Rb = sR[bo][n];
            if (Ra == kNone || Rb == kNone) continue;
            const double val = i64_scaled_to_double(acc[j][v], Ra + Rb - 8 * LMAX);
            if (val == 0.0) continue;
            atomicAdd(&g.G[(int64_t)gm * g.n_cols + gn], val);
            if (SYM && gm != gn) atomicAdd(&g.G[(int64_t)gn * g.n_cols + gm], val);
        }
}

template <int SA, int SB, int LMAX, bool SYM, bool SAME, int KW, bool NAT>
cudaError_t launch_tc(const GramTcArgs& g, cudaStream_t s) {
    constexpr size_t smem = (size_t)(SA + SB) * kST * KW * 2;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<SA, SB, LMAX, SYM, SAME, KW, NAT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gram_tc_kernel<SA, SB, LMAX, SYM, SAME, KW, NAT><<<(unsigned)g.n_items, kThreads, smem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_tc(const GramTcArgs& g, GramMode mode, cudaStream_t s) {
    if (g.n_items == 0) return cudaSuccess;
    // P^T Y: 3 slices (the lower two natural bf16), levels <= 4, windows of
    // 128 rows (the level-2 window sums stay below 2^23); P^T P: 5 slices on
    // the fixed grid, levels <= 6, windows of 64 rows (shared memory for 10
    // staged slices).  The symmetric modes take the upper super-tiles only
    // and mirror them.
    switch (mode) {
        case GramMode::PtP: return launch_tc<5, 5, 6, true, true, 64, false>(g, s);
        case GramMode::PtYSym: return launch_tc<3, 3, 4, true, false, 128, true>(g, s);
        default: return launch_tc<3, 3, 4, false, false, 128, true>(g, s);
    }
}

int gram_tc_tile() { return kST; }
int gram_tc_split_rows() { return 1024; }

}  // namespace femf
