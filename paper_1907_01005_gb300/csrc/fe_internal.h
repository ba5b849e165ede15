// Internal declarations shared by the host builder (host.cpp) and the CUDA
// kernels (apply.cu, gram.cu).  Nothing here is part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fe_mf.h"

namespace femf {

constexpr int kMaxP = 4;            // highest degree with GPU kernels
constexpr int kMaxN = kMaxP + 1;    // 1D points per cell
constexpr int kMaxW = 16;           // widest column block

// 1D operators of the sum-factorised cell kernel on the reference cell
// [0,1]^3 with n = p+1 Gauss points per direction (Sec. 3.2):
//   S[q][a]  = l_a(x_q)              nodal basis (GLL nodes) at Gauss point q
//   Sb[a][q] = S[q][a] * w_q         transposed interpolation with the weight
//   A[d][l][m] = c_d (D^T W D)[l][m] / w_l,  c_d = |J| / (2 h_d^2)
// where D is the collocation derivative on the Gauss points.  With these, the
// cell operator on nodal values u reads
//   y = Sb^3 [ sum_d A_d u_q + |J| V_q u_q ],   u_q = S^3 u,
// the weights w_i w_j w_k of the tensor rule being folded into Sb and A.
template <typename T>
struct CellConsts {
    T S[kMaxN][kMaxN];
    T Sb[kMaxN][kMaxN];
    T A[3][kMaxN][kMaxN];
    T jxw;       // |J| = hx hy hz
    // Variant used by the register-resident kernel, which takes V unscaled:
    // A / |J| in A above and |J| Sb here, for the first of the three
    // transposed interpolations only (the other two use Sb).
    T Sb1[kMaxN][kMaxN];
};

// One (patch, column block) work item of the apply.  Slot b = dx + 2 dy + 4 dz
// names the row block of patch (px - 1 + dx, py - 1 + dy, pz - 1 + dz); off[b]
// is the element offset of block (that row block, column block) in the value
// array, or -1 when the block is not stored (or the patch does not exist).
// Halo slots of the apply's write (unit_common.cuh): slot (block (r, c), e)
// holds the contributions of patch r + e (e = ex + 2 ey + 4 ez != 0, an
// upper neighbour of r) to the rows of block (r, c) on r's face with mask e,
// as rows of the block's row stride, in the face order of halo_face_index.
// hout[s] (s != 7): the slot this patch writes for the block of slot s;
// hin[e]: the slots (own block, e) this patch reads.  Offsets in 16-byte
// units from the start of the halo region, -1 where there is none.
struct Tile {
    int64_t off[8];
    int32_t hout[8];
    int32_t hin[8];
    int32_t patch;      // rank of the patch (= its row block)
    int32_t pxyz;       // px | py << 10 | pz << 20
    int32_t width;      // column block width
    int32_t cellmask;   // bit c (c = cx + 2 cy + 4 cz) set iff that cell touches a stored block
    int32_t ld;         // row stride of the column block's blocks (elements)
    int32_t pad;
};

// Packed work unit of the register-resident apply (p <= 2): one patch and up
// to four of its column blocks with at most 32 columns in total; CTA lane j
// takes column j of the concatenated blocks.  off[b][s] is the offset of
// block (row block of slot s, column block b) in units of 16 bytes, or -1.
constexpr int kUnitBlocks = 4;
constexpr int kUnitLanes = 32;
constexpr int kUnitLdSum = 36;    // sum of the blocks' row strides in a unit
struct Unit {
    int32_t off[kUnitBlocks][8];
    int32_t hout[kUnitBlocks][8];   // halo slots written (see Tile), per block and slot
    int32_t hin[kUnitBlocks][8];    // halo slots read, per block and upper-neighbour offset e
    int32_t patch;      // rank of the patch
    int32_t pxyz;       // px | py << 10 | pz << 20
    int32_t nb;         // column blocks in the unit
    int32_t width[kUnitBlocks];
    int32_t ld[kUnitBlocks];
    int32_t cellmask[kUnitBlocks];
    int32_t pad;
};

// Gram work: entries are (block of A, block of B, rows) for one column-block
// pair and one row block; items are contiguous entry ranges of one pair.
struct GramEntry {
    int64_t offA;
    int64_t offB;
    int32_t rows;
    int32_t pad;
};
struct GramItem {
    int32_t c1, c2;
    int32_t begin, end;
};

// Tensor-core Gram of FP32 multivectors (gram_tc.cu): work is grouped by
// runs of consecutive row blocks; a group's union of column blocks is laid
// out as `width` dense columns, its output tiled gram_tc_tile() square and
// its rows split into items of at most gram_tc_item_rows().
constexpr int kMaxGroup = 8;     // row blocks per group
constexpr int kMaxUnion = 64;    // column blocks in a group's union
struct GramTcGroup {
    int32_t r0, r1;     // row blocks [r0, r1)
    int32_t k_rows;     // rows of the group
    int32_t n_u;        // column blocks in the union
    int32_t width;      // columns of the union
    int32_t u_base;     // offset of the group's (r1-r0) x n_u block-offset table
    int32_t c_base;     // offset of the group's column tables
    int32_t pad;
};
struct GramTcItem {
    int32_t group;
    int32_t tile;       // mi | ni << 16 (square tiles of gram_tc_tile() union columns)
    int32_t k0, k1;     // rows [k0, k1) of the group (at most gram_tc_item_rows())
};
struct GramTcArgs {
    const float* A;
    const float* B;
    const GramTcGroup* groups;
    const GramTcItem* items;
    int64_t n_items;
    int64_t n_items_diag;       // P^T P: the first n_items_diag items are diagonal tiles (mi == ni)
    const int64_t* union_off;   // element offset of block (row block, union slot) or -1
    const int32_t* col_info;    // (slot << 16) | (column in block << 8) | row stride of the block
    const int32_t* col_glob;    // global column id
    const int32_t* rows;        // rows of each row block
    int16_t* item_exp;          // scratch: item exponents, 2 x gram_tc_tile() per item (A side, B side)
    int32_t sm_limit;           // > 0: the persistent kernel runs on at most this many SMs
    int32_t n_cols;
    double* G;
    int32_t* status;            // device status word (set on a malformed work item)
};
// PtY: full A^T B; PtP: A^T A on upper super-tiles, mirrored; PtYSym: A^T B
// known to be symmetric (closed pattern), upper super-tiles, mirrored
enum class GramMode { PtY = 0, PtP = 1, PtYSym = 2 };
cudaError_t launch_gram_tc(const GramTcArgs& a, GramMode mode, cudaStream_t s);
// SMs a persistent launch may occupy: the device's, capped by sm_limit > 0
int usable_sms(int32_t sm_limit);
int gram_tc_tile();         // output tile edge of the tensor-core Gram (union columns)
int gram_tc_item_rows(bool pp);   // most rows of a work item of P^T P (pp) or P^T Y

template <typename T>
struct ApplyArgs {
    const T* P;
    T* Y;
    const T* Vq;
    const Tile* tiles;
    int64_t n_tiles;
    int32_t npx, npy, npz;
    int32_t lx, ly, lz;
    int32_t dirichlet;
    int32_t wmax;             // widest column block (columns per cell round)
    int32_t ldmax;            // largest row stride (a multiple of 16 bytes): row stride capacity of
                              // the patch tensors in shared memory
    int32_t cells_per_round;  // cells processed concurrently (1, 2, 4 or 8)
    unsigned long long* ticket;   // work counter (zeroed before the launch): tiles go in descending order
    int32_t* done;            // tiles per patch whose halo is written (zeroed before the launch), by patch id
    const int32_t* count;     // tiles per patch, by patch id
    T* halo;                  // halo region (Tile.hout / hin offsets)
    int32_t* status;          // device status word (0 = ok)
    int32_t mass;             // 1: the mass operator (no gradient term, V = 1; Vq unused)
    CellConsts<T> k;
};

template <typename T>
struct GramArgs {
    const T* A;
    const T* B;
    const GramEntry* entries;
    const GramItem* items;
    int64_t n_items;
    const int32_t* cb_ptr;
    const int32_t* ld;        // row stride of each column block
    int32_t n_cols;
    int32_t symmetric;        // 1: also write the mirrored block for c1 != c2
    double* G;
};

// Launchers (apply.cu / gram.cu).  They return a cudaError_t and leave the
// message to the caller.
template <typename T>
cudaError_t launch_apply(int p, const ApplyArgs<T>& a, cudaStream_t s);
template <typename T>
struct ApplyUnitArgs {
    const T* P;
    T* Y;
    const T* Vq;
    const Unit* units;
    int64_t n_units;
    unsigned long long* ticket;   // work counter (zeroed before the launch): units go in descending order
    int32_t persistent;           // 1: ctas_per_sm CTAs per SM loop over the work counter; 0: a CTA per unit
    int32_t ctas_per_sm;
    int32_t sm_limit;             // > 0: the persistent launch occupies at most this many SMs' worth
    int32_t* done;                // units per patch whose halo is written (zeroed before the launch), by patch id
    const int32_t* count;         // units per patch, indexed by patch id
    T* halo;                      // halo region (Unit.hout / hin offsets)
    int32_t npx, npy, npz;
    int32_t lx, ly, lz;
    int32_t dirichlet;
    int32_t* status;
    int32_t mass;                 // 1: the mass operator (no gradient term, V = 1; Vq unused)
    CellConsts<T> k;
};
template <typename T>
cudaError_t launch_apply_units(int p, const ApplyUnitArgs<T>& a, cudaStream_t s);

// Cell-matrix form of the apply (apply_cellmat.cu; p <= 2, FP32, tensor
// cores).  Constant operands per operator ("set"): B1 = [K_L; S3] (H) or
// [M_c; 0] (M), 2 npad rows, and B2 = Sb3 with |J| (H) or 0 (M), npad rows;
// each row holds 32 FP32 values (cell nodes or Gauss points, zero-padded) in
// the 128-byte-swizzled K-major tile layout of the kernel's shared memory:
// element (r, k) at float index 32 r + 4 ((k / 4) ^ (r % 8)) + k % 4.  A set
// is B1 high, B1 low, B2 high, B2 low, the high part the TF32 rounding of
// the matrix and the low part the FP32 remainder.
constexpr int cellmat_npad(int p) { return p == 1 ? 16 : 32; }
constexpr int cellmat_set_floats(int p) { return 6 * cellmat_npad(p) * 32; }
struct CellMatArgs {
    const float* P;
    float* Y;
    const float* Vq;
    const Unit* units;
    int64_t n_units;
    unsigned long long* ticket;   // work counter, zeroed before the launch (CTAs are persistent)
    int32_t* done;                // units per patch whose halo is written (zeroed before the launch), by patch id
    const int32_t* count;         // units per patch, by patch id
    float* halo;                  // halo region (Unit.hout / hin offsets)
    int32_t npx, npy, npz;
    int32_t lx, ly, lz;
    int32_t dirichlet;
    int32_t* status;
    int32_t mass;                 // 1: the mass operator (stage 1 only, Vq unused)
    const float* consts;          // the operator's constant set (16-byte aligned, device)
    int32_t sm_limit;             // > 0: at most this many SMs' worth of persistent CTAs
};
cudaError_t launch_apply_cellmat(int p, const CellMatArgs& a, cudaStream_t s);
template <typename T>
size_t apply_smem_bytes(int p, int wmax, int ldmax, int cells_per_round);
template <typename T>
int apply_threads(int p, int wmax, int cells_per_round);
int apply_max_threads(int p);
template <typename T>
cudaError_t launch_gram(const GramArgs<T>& a, cudaStream_t s);

// Post-multiplication C = alpha (A X + gamma A) + beta C (mmult.cu, Alg. 7)
struct MmultItem {
    int32_t r;          // row block
    int32_t i0, j0;     // first row of the chunk, first union column of the output chunk
    int32_t pad;
};
// A stored block as the tensor-core post-multiplication maps it into its row
// block's padded union: one record per block, in CSR order
struct MmBlock {
    int64_t off;        // element offset of the block
    int32_t u0;         // first padded-union column
    int32_t ld;         // row stride (padded width)
    int32_t w;          // width
    int32_t gcol0;      // first global column
    int32_t pcol0;      // first padded global column
    int32_t pad;
};
template <typename T>
struct MmultArgs {
    const T* A;
    T* C;
    const double* X;            // M x M, row-major, the multivectors' column order
    const T* Xw;                // X in the working precision (set by launch_mmult)
    int32_t n_cols;
    int32_t wmax_union;         // largest padded union (row strides of a row block's stored blocks)
    const MmultItem* items;
    int64_t n_items;
    const int64_t* row_ptr;     // BCSR pattern on the device
    const int32_t* col_idx;
    const int64_t* blk_off;
    const int32_t* cbp;
    const int32_t* ld;
    const int32_t* rb_rows;
    const int32_t* ucol0;       // first padded-union column of each stored block within its row block
    const int32_t* rb_union;    // padded-union columns of each row block
    // tensor-core path (FP32): padded global columns (each column block at
    // pcol0[c], ld columns), their global ids (-1 = padding), and X^T in
    // padded coordinates, split into TF32 high parts and remainders (set by
    // launch_mmult_tc)
    const int32_t* pcol0;
    const int32_t* pglob;
    const MmBlock* mm_blocks;
    int32_t n_pcols;
    const float* XThi;
    const float* XTlo;
    int32_t sm_limit;           // > 0: at most this many SMs' worth of persistent CTAs (tensor-core path)
    double alpha, gamma, beta;
    int32_t* status;
};
template <typename T>
struct TraceArgs {
    const T* D;
    const T* G;
    int64_t n_blocks;
    const int32_t* block_rb;    // row block of each stored block
    const int32_t* col_idx;
    const int64_t* blk_off;
    const int32_t* cbp;
    const int32_t* ld;
    const int32_t* rb_rows;
    double* out;                // accumulated with atomics (zeroed by the caller)
};
template <typename T>
size_t mmult_smem_bytes(int wmax_union);
// Dynamic shared memory the post-multiplication may use (two k-tile buffers
// and the union tables); x_round (FP32 only) receives X rounded to FP32.
constexpr size_t kMmultSmemMax = 200 * 1024;
template <typename T>
cudaError_t launch_mmult(const MmultArgs<T>& a, float* x_round, cudaStream_t s);
// FP32 on the tensor cores (mmult_tc.cu); xt holds 2 n_pcols^2 floats
size_t mmult_tc_smem_bytes(int wmax_union);
constexpr size_t kMmultTcSmemMax = 55 * 1024;    // four CTAs per SM
cudaError_t launch_mmult_tc(const MmultArgs<float>& a, float* xt, cudaStream_t s);
template <typename T>
cudaError_t launch_trace(const TraceArgs<T>& a, cudaStream_t s);

// *sink_ok: the first and last CTA slot of the sink hold thread 0's chain sum
// as the host computes it
cudaError_t probe_fma(int dtype, int64_t iters, double* flops_per_s, cudaStream_t s, bool* sink_ok);
constexpr int kProbeSinkSlots = 4096;   // per-CTA slots of the allocation-free probe (512 SMs x 8)
// *too_many: 0 = ran; > 0 = the device needs that many slots (> kProbeSinkSlots);
// -1 = device ordinal beyond the per-device table; -2 = the static sink,
// read back through its symbol, does not hold the chain sums
cudaError_t probe_fma_static(int dtype, int64_t iters, double* flops_per_s, cudaStream_t s, int* too_many);

// Device status codes written by kernels.
enum DeviceStatus : int32_t {
    kDevOk = 0,
    kDevBadTile = 1,
    kDevTimeout = 2,      // a bounded wait on the tensor cores ran out
};

}  // namespace femf
