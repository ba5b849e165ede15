// Gram products of FP32 multivectors on the tensor cores with an error-free
// split (C = A^T B over stored blocks, Alg. 8; FP64-accurate accumulation).
//
// Every FP32 value of a column m of the group slab is written as a sum of S
// slices q_s 2^(E_m - 8 s) with integers |q_s| <= 256 (exact in bf16), E_m a
// power-of-two bound of the column's magnitude over the group's rows.  Then
//   sum_k a_km b_kn = sum_{s,t} 2^(E_m + F_n - 8(s+t)) sum_k q_s,km r_t,kn ,
// and each inner sum over a window of <= 64 rows is an integer below 2^23, so
// the bf16 x bf16 -> FP32 tensor-core accumulation is exact.  Slice pairs of
// the same level L = s + t share a scale; levels above the cut-off LMAX are
// dropped.  Every level is summed on the tensor cores over a window of 64
// rows only (each window sum is an integer below 2^23, exact whatever the
// rounding of the tensor-core adder), then the levels are combined into one
// int64 per output element (level L shifted by 8 (LMAX - L) bits), so the
// sum over the group is exact.  Running FP32 sums over the whole group are
// avoided on purpose: the tensor-core FP32 accumulation does not round to
// nearest, and its bias over thousands of rows reaches 1e-10 of the result.
// The int64 is converted to FP64 with integer operations only (the FP64 pipe
// of this GPU runs at 1/64 of the FP32 rate) and added into the dense FP64
// result with one atomic per output element and row-block group.
//
// Work item: (group of consecutive row blocks, 48 x 48 output tile of the
// group's union columns); 6 warps in a 3 x 2 layout, each owning a 16 x 24
// sub-tile (three m16n8k16 tiles).
#include <cuda_bf16.h>

#include "fe_internal.h"

namespace femf {
namespace {

constexpr int kTile = 48;        // output tile edge (union columns)
constexpr int kWarpsM = 3, kWarpsN = 2;
constexpr int kThreads = 32 * kWarpsM * kWarpsN;
constexpr int kNT = 3;           // n8 tiles per warp (16 x 24 sub-tile)
constexpr int kChunk = 32;       // rows staged per iteration
constexpr int kRowWords = 20;    // 32-bit words per staged column (16 used: 32 rows of bf16)
constexpr int kFlushRows = 64;   // rows per exact window (window sums < 2^23)
constexpr int kMaxRows = (2 * kMaxP + 1) * (2 * kMaxP + 1) * (2 * kMaxP + 1);   // rows of a row block

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// word index of (column row, word kw = k/2) in a staged slice, XOR-swizzled
// so that 32 consecutive columns with the same kw hit 32 different banks and
// the fragment loads (8 columns x 4 words) stay conflict-free
__device__ __forceinline__ int swz(int col, int kw) { return col * kRowWords + (kw ^ ((col >> 3) & 3)); }

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

// slices of two rows (x0, x1) of one column, already normalised to |x| < 1:
// q_s = rint(r 2^(8s)), r -= q_s 2^(-8s); stored as packed bf16 pairs
template <int S>
__device__ __forceinline__ void slice_store(uint32_t* base, int slice_words, int word, float x0, float x1) {
#pragma unroll
    for (int s = 1; s <= S; ++s) {
        const float up = __int_as_float((127 + 8 * s) << 23);   // 2^(8s)
        const float dn = __int_as_float((127 - 8 * s) << 23);   // 2^(-8s)
        const float q0 = rintf(x0 * up), q1 = rintf(x1 * up);
        x0 = fmaf(-q0, dn, x0);
        x1 = fmaf(-q1, dn, x1);
        const __nv_bfloat162 v = __floats2bfloat162_rn(q0, q1);
        base[(s - 1) * slice_words + word] = *reinterpret_cast<const uint32_t*>(&v);
    }
}

template <int SA, int SB, int LMAX, bool SYM>
__global__ void __launch_bounds__(kThreads) gram_tc_kernel(const GramTcArgs g) {
    constexpr int NLEV = LMAX - 1;                 // levels 2..LMAX
    constexpr int SW = kTile * kRowWords;          // words per staged slice
    __shared__ __align__(16) uint32_t As[SA * SW];
    __shared__ __align__(16) uint32_t Bs[SB * SW];
    __shared__ int sEa[kTile], sEb[kTile];
    __shared__ float sNa[kTile], sNb[kTile];
    __shared__ unsigned sMaxA[kTile], sMaxB[kTile];
    __shared__ int64_t sOff[kMaxGroup * kMaxUnion];
    __shared__ int sColA[kTile], sColB[kTile];     // (u << 16) | (a << 8) | w, or -1
    __shared__ int sGcolA[kTile], sGcolB[kTile];
    __shared__ int sRowRb[kChunk], sRowLoc[kChunk];
    __shared__ int sPref[kMaxGroup + 1];

    const GramTcItem it = g.items[blockIdx.x];
    const GramTcGroup gr = g.groups[it.group];
    const int mi = it.tile & 0xffff, ni = it.tile >> 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrb = gr.r1 - gr.r0;
    // Work-list check: a group has 1..kMaxGroup row blocks and at most kMaxUnion
    // union columns (the shared tables and the int64 bound depend on it); a
    // malformed item sets the status word and leaves G untouched.
    if (nrb < 1 || nrb > kMaxGroup || gr.n_u < 1 || gr.n_u > kMaxUnion || gr.width < 1 ||
        gr.width > kMaxUnion * kMaxW || gr.k_rows > kMaxGroup * kMaxRows || mi * kTile >= gr.width || ni * kTile >= gr.width) {
        if (tid == 0 && g.status) atomicExch(g.status, kDevBadTile);
        return;
    }

    // ---- group tables ------------------------------------------------------
    for (int e = tid; e < nrb * gr.n_u; e += kThreads) sOff[e] = g.union_off[gr.u_base + e];
    if (tid < kTile) {
        const int ma = mi * kTile + tid, nb = ni * kTile + tid;
        sColA[tid] = ma < gr.width ? g.col_info[gr.c_base + ma] : -1;
        sGcolA[tid] = ma < gr.width ? g.col_glob[gr.c_base + ma] : -1;
        sColB[tid] = nb < gr.width ? g.col_info[gr.c_base + nb] : -1;
        sGcolB[tid] = nb < gr.width ? g.col_glob[gr.c_base + nb] : -1;
        sMaxA[tid] = 0u;
        sMaxB[tid] = 0u;
    }
    if (tid == 0) {
        sPref[0] = 0;
        for (int r = 0; r < nrb; ++r) sPref[r + 1] = sPref[r] + g.rows[gr.r0 + r];
    }
    __syncthreads();

    // ---- pass 1: column magnitude bounds (|x| < 2^E) over the group --------
    {
        const int col = tid % kTile, ph = tid / kTile, nph = kThreads / kTile;
        const int ca = sColA[col], cb = sColB[col];
        float ma = 0.f, mb = 0.f;
        for (int r = 0; r < nrb; ++r) {
            const int rows = sPref[r + 1] - sPref[r];
            if (ca >= 0) {
                const int64_t o = sOff[r * gr.n_u + (ca >> 16)];
                const int a = (ca >> 8) & 0xff, w = ca & 0xff;
                if (o >= 0)
                    for (int k = ph; k < rows; k += nph) ma = fmaxf(ma, fabsf(g.A[o + (int64_t)k * w + a]));
            }
            if (cb >= 0) {
                const int64_t o = sOff[r * gr.n_u + (cb >> 16)];
                const int a = (cb >> 8) & 0xff, w = cb & 0xff;
                if (o >= 0)
                    for (int k = ph; k < rows; k += nph) mb = fmaxf(mb, fabsf(g.B[o + (int64_t)k * w + a]));
            }
        }
        atomicMax(&sMaxA[col], __float_as_uint(ma));   // non-negative floats order as unsigned
        atomicMax(&sMaxB[col], __float_as_uint(mb));
    }
    __syncthreads();
    if (tid < kTile) {
        const float ma = __uint_as_float(sMaxA[tid]), mb = __uint_as_float(sMaxB[tid]);
        const int ea = ma > 0.f ? ilogbf(ma) + 1 : 0, eb = mb > 0.f ? ilogbf(mb) + 1 : 0;
        sEa[tid] = ea;
        sEb[tid] = eb;
        sNa[tid] = ma > 0.f ? scalbnf(1.0f, -ea) : 0.f;
        sNb[tid] = mb > 0.f ? scalbnf(1.0f, -eb) : 0.f;
    }
    __syncthreads();

    // ---- pass 2: sliced products over row chunks ----------------------------
    float wacc[NLEV][kNT][4];         // window sums of each level (exact integers)
    // all levels combined, exact over the group: a group has at most kMaxGroup
    // row blocks of <= kMaxRows = 729 rows, i.e. <= 92 windows; a level-2
    // window sum is <= 64 * 2^16 = 2^22 and is shifted by 8 (LMAX - 2) <= 32
    // bits (the other levels add less than 2^-7 of that), so |acc| < 2^61
    long long acc[kNT][4];
#pragma unroll
    for (int j = 0; j < kNT; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            acc[j][v] = 0;
#pragma unroll
            for (int l = 0; l < NLEV; ++l) wacc[l][j][v] = 0.f;
        }
    const int wm = (warp / kWarpsN) * 16, wn = (warp % kWarpsN) * (8 * kNT);
    const int gid = lane >> 2, tig = lane & 3;
    const bool wact = (mi * kTile + wm < gr.width) && (ni * kTile + wn < gr.width) &&
                      (!SYM || mi < ni || wm < wn + 8 * kNT);   // skip sub-tiles beyond the union

    int since_flush = 0;
    for (int k0 = 0; k0 < gr.k_rows; k0 += kChunk) {
        if (tid < kChunk) {
            const int k = k0 + tid;
            int r = -1, loc = 0;
            if (k < gr.k_rows) {
                r = 0;
                while (k >= sPref[r + 1]) ++r;
                loc = k - sPref[r];
            }
            sRowRb[tid] = r;
            sRowLoc[tid] = loc;
        }
        __syncthreads();
        // stage: each thread takes (column, pair of rows)
        for (int e = tid; e < kTile * (kChunk / 2); e += kThreads) {
            const int col = e % kTile, kw = e / kTile;
            float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
            const int ca = sColA[col], cb = sColB[col];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = sRowRb[2 * kw + h];
                if (r < 0) continue;
                const int loc = sRowLoc[2 * kw + h];
                if (ca >= 0) {
                    const int64_t o = sOff[r * gr.n_u + (ca >> 16)];
                    if (o >= 0) (h ? a1 : a0) = g.A[o + (int64_t)loc * (ca & 0xff) + ((ca >> 8) & 0xff)];
                }
                if (cb >= 0) {
                    const int64_t o = sOff[r * gr.n_u + (cb >> 16)];
                    if (o >= 0) (h ? b1 : b0) = g.B[o + (int64_t)loc * (cb & 0xff) + ((cb >> 8) & 0xff)];
                }
            }
            const int wd = swz(col, kw);
            slice_store<SA>(As, SW, wd, a0 * sNa[col], a1 * sNa[col]);
            slice_store<SB>(Bs, SW, wd, b0 * sNb[col], b1 * sNb[col]);
        }
        __syncthreads();
        if (wact) {
#pragma unroll
            for (int kk = 0; kk < kChunk / 2; kk += 8) {     // 16 rows = 8 words per k-step
                uint32_t af[SA][4];
                const int r0 = wm + gid, r1 = wm + gid + 8;
#pragma unroll
                for (int s = 0; s < SA; ++s) {
                    af[s][0] = As[s * SW + swz(r0, kk + tig)];
                    af[s][1] = As[s * SW + swz(r1, kk + tig)];
                    af[s][2] = As[s * SW + swz(r0, kk + 4 + tig)];
                    af[s][3] = As[s * SW + swz(r1, kk + 4 + tig)];
                }
#pragma unroll
                for (int j = 0; j < kNT; ++j) {
                    const int n = wn + 8 * j + gid;
                    uint32_t bf[SB][2];
#pragma unroll
                    for (int t = 0; t < SB; ++t) {
                        bf[t][0] = Bs[t * SW + swz(n, kk + tig)];
                        bf[t][1] = Bs[t * SW + swz(n, kk + 4 + tig)];
                    }
#pragma unroll
                    for (int s = 1; s <= SA; ++s)
#pragma unroll
                        for (int t = 1; t <= SB; ++t) {
                            const int L = s + t;
                            if (L > LMAX) continue;
                            mma_bf16(wacc[L - 2][j], af[s - 1], bf[t - 1][0], bf[t - 1][1]);
                        }
                }
            }
        }
        since_flush += kChunk;
        if (since_flush >= kFlushRows) {
#pragma unroll
            for (int j = 0; j < kNT; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
#pragma unroll
                    for (int l = 0; l < NLEV; ++l) {
                        acc[j][v] += (long long)__float2int_rn(wacc[l][j][v]) << (8 * (NLEV - 1 - l));
                        wacc[l][j][v] = 0.f;
                    }
                }
            since_flush = 0;
        }
        __syncthreads();
    }
    if (!wact) return;

    // ---- epilogue: levels -> int64 -> FP64, one atomic per element ----------
#pragma unroll
    for (int j = 0; j < kNT; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int m = wm + gid + (v >= 2 ? 8 : 0);
            const int n = wn + 8 * j + tig * 2 + (v & 1);
            const int gm = sGcolA[m], gn = sGcolB[n];
            if (gm < 0 || gn < 0) continue;
            if (SYM && mi == ni && m > n) continue;      // lower half of a diagonal tile: mirrored below
            long long t = acc[j][v];
#pragma unroll
            for (int l = 0; l < NLEV; ++l) t += (long long)__float2int_rn(wacc[l][j][v]) << (8 * (NLEV - 1 - l));
            const double val = i64_scaled_to_double(t, sEa[m] + sEb[n] - 8 * LMAX);
            if (val == 0.0) continue;
            atomicAdd(&g.G[(int64_t)gm * g.n_cols + gn], val);
            if (SYM && gm != gn) atomicAdd(&g.G[(int64_t)gn * g.n_cols + gm], val);
        }
}

}  // namespace

cudaError_t launch_gram_tc(const GramTcArgs& g, bool sym, cudaStream_t s) {
    if (g.n_items == 0) return cudaSuccess;
    // The error is set by the residual after the last slice (|r| <= 2^(-8S-1)
    // of the column bound) and by the first dropped level (<= 2^(-8 LMAX + 14)
    // per product), so LMAX = S + 1 balances the two.  P^T Y: 3 slices, levels
    // <= 4 (6 products, ~2^-25 of the result); P^T P: 5 slices, levels <= 6
    // (15 products, ~2^-40: columns whose values span many binades within a
    // group, as orbitals decaying across a p = 4 patch do, stay well inside
    // a 1e-10 normwise bound).
    if (sym)
        gram_tc_kernel<5, 5, 6, true><<<(unsigned)g.n_items, kThreads, 0, s>>>(g);
    else
        gram_tc_kernel<3, 3, 4, false><<<(unsigned)g.n_items, kThreads, 0, s>>>(g);
    return cudaGetLastError();
}

int gram_tc_tile() { return kTile; }

}  // namespace femf
