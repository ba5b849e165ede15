/*
 * fe_mf.h -- C ABI of the GB300 matrix-free BCSR Hamiltonian library.
 *
 * The library applies the finite-element Hamiltonian H = -1/2 Laplacian + V(x)
 * (Sec. 2; Eq. fe_matrices, Sec. 3.1) matrix-free to a block-sparse (BCSR)
 * multivector P of localised orbitals on a box mesh of hexahedral Q_p cells,
 * giving Y = H P restricted to P's block pattern (Alg. 6, Sec. 3.5), and forms
 * the Gram products P^T Y and P^T P (Alg. 8, Sec. 3.6; Eqs. inner1/inner2).
 *
 * Conventions that hold for every entry point
 * -------------------------------------------
 * - Every function returns an int status: FE_OK (0) or a negative FE_E* code.
 *   On error a message is stored in a thread-local buffer, readable with
 *   fe_last_error().  No function aborts the process.
 * - Handles (fe_mesh, fe_bcsr) are opaque, created and destroyed by the
 *   library.  They are not thread-safe: one handle is used by one host
 *   thread at a time.
 * - Device memory is owned by the caller.  Entry points that take a device
 *   pointer document how long the library keeps it: a pointer passed to a
 *   *_bind / *_upload / fe_mesh_set_potential call is kept by the handle until
 *   the handle is destroyed or re-bound, and must stay valid that long.
 * - `stream` is a cudaStream_t (CUstream) passed as void*; NULL means the
 *   legacy default stream.  Device work is enqueued on it and the call returns
 *   without synchronising, unless a function says otherwise.
 * - Host arrays are read during the call only and never kept.
 *
 * Mesh, numbering and blocking
 * ----------------------------
 * The mesh is a box of nx*ny*nz axis-aligned cells of edge hx*hy*hz with
 * Lagrange Q_p elements; nodes sit on the lattice (p nx + 1)(p ny + 1)(p nz + 1)
 * at x = h (cell + xi_k), xi the Gauss-Lobatto-Legendre points on [0,1].
 * Row blocks follow Alg. 1 with 2x2x2-cell patches as the coarse cells:
 * patches are ordered along a Morton curve (x in the lowest bit of each bit
 * triple), and row block r holds the nodes of the patch of rank r that no
 * earlier patch holds, i.e. every node belongs to the component-wise lowest
 * patch that contains it.  Inside a row block, DoFs are numbered
 * lexicographically (x fastest) over the patch-local lattice.
 * Homogeneous Dirichlet (dirichlet=1): boundary nodes keep their DoF ids; the
 * operator treats their input values as zero and writes zero to their rows.
 */
#ifndef FE_MF_H
#define FE_MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FE_OK 0
#define FE_EINVAL (-1)      /* an argument is out of range or NULL */
#define FE_ENOMEM (-2)      /* host allocation failed, or a buffer is too small */
#define FE_EPATTERN (-3)    /* a block pattern is malformed or two patterns differ */
#define FE_ECUDA (-4)       /* a CUDA runtime call failed (message has the CUDA error) */
#define FE_EDEVICE (-5)     /* a kernel reported an error through the device status word */
#define FE_ESTATE (-6)      /* the handle is not in the state the call needs (e.g. not bound) */
#define FE_EUNSUPPORTED (-7)/* valid but not supported by this build (e.g. degree p > 4 on the GPU) */

#define FE_F32 1            /* FP32 storage, FP32 cell arithmetic, FP64 Gram accumulation */
#define FE_F64 2            /* FP64 storage and arithmetic throughout */

/* Forms of the cell operator (fe_bcsr_set_form) */
#define FE_FORM_SUMFAC 0    /* sum factorisation on the FP32/FP64 ALUs (Sec. 3.5, Alg. 6) */
#define FE_FORM_CELLMAT 1   /* element matrices as dense products on the tensor cores (Sec. 3.2) */

typedef struct fe_mesh fe_mesh;
typedef struct fe_bcsr fe_bcsr;

/* Library version (major*10000 + minor*100 + patch). */
int fe_version(void);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to n bytes).  Returns FE_OK. */
int fe_last_error(char* buf, size_t n);

/* ------------------------------------------------------------------------
 * Mesh and DoF map (Sec. 3.1; Alg. 1)
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny, nz;           /* cells per direction (even) */
    int32_t p;                    /* polynomial degree */
    int32_t dirichlet;            /* 1: homogeneous Dirichlet on all six faces */
    int32_t npx, npy, npz;        /* patches (row blocks) per direction */
    int32_t lx, ly, lz;           /* lattice nodes per direction */
    int32_t n_row_blocks;         /* = npx*npy*npz */
    int32_t max_rows_per_block;   /* largest row block */
    int32_t nq1;                  /* Gauss points per direction (= p+1) */
    int64_t n_dofs;               /* = lx*ly*lz */
    int64_t n_cells;
    int64_t n_q;                  /* quadrature points = n_cells * nq1^3 */
    double hx, hy, hz;
} fe_mesh_info_t;

/* Creates the box mesh, its patch order and DoF numbering (Alg. 1 reading
 * above).  nx, ny, nz: even, >= 2; h*: > 0; p: 1..6 on the host, 1..4 on the
 * GPU; dirichlet: 0 or 1.  FE_EINVAL on bad arguments. */
int fe_mesh_create(int32_t nx, int32_t ny, int32_t nz, double hx, double hy, double hz,
                   int32_t p, int32_t dirichlet, fe_mesh** out);
int fe_mesh_destroy(fe_mesh* mesh);
int fe_mesh_get_info(const fe_mesh* mesh, fe_mesh_info_t* info);

/* rb_ptr[n_row_blocks+1]: DoFs of row block r are [rb_ptr[r], rb_ptr[r+1]). */
int fe_mesh_row_blocks(const fe_mesh* mesh, int64_t* rb_ptr);

/* pxyz[3*n_row_blocks]: patch coordinates (px, py, pz) of row block r. */
int fe_mesh_patch_coords(const fe_mesh* mesh, int32_t* pxyz);

/* ijk[3*n_dofs]: lattice coordinates (I, J, K) of each DoF id. */
int fe_mesh_dof_keys(const fe_mesh* mesh, int32_t* ijk);

/* xyz[3*n_dofs]: physical coordinates of each DoF id (FP64). */
int fe_mesh_node_coords(const fe_mesh* mesh, double* xyz);

/* xyz[3*n_q]: physical Gauss points in the potential layout
 * [row block r][cell c = cx + 2 cy + 4 cz of the patch][qz][qy][qx]. */
int fe_mesh_quad_points(const fe_mesh* mesh, double* xyz);

/* Bytes of device workspace the mesh needs: the device status word and, for
 * p <= 2, the constant operands of the cell-matrix form (48 KB at p = 2). */
int fe_mesh_workspace_bytes(const fe_mesh* mesh, size_t* bytes);

/* Copies the mesh tables into the caller's device buffer `workspace_dev`
 * (at least fe_mesh_workspace_bytes, 256-byte aligned) on `stream` and keeps
 * the pointer.  FE_ENOMEM if `bytes` is too small; FE_ECUDA on copy failure. */
int fe_mesh_upload(fe_mesh* mesh, void* workspace_dev, size_t bytes, void* stream);

/* Registers the potential V at the Gauss points (Eq. fe_matrices: the
 * N_i V N_j term): n_q values of type dtype (FE_F32 or FE_F64) on the device,
 * in the layout of fe_mesh_quad_points.  The pointer is kept; one potential of
 * each dtype can be registered. */
int fe_mesh_set_potential(fe_mesh* mesh, const void* vq_dev, int32_t dtype);

/* Reads and clears the device status word on `stream` (synchronises it).
 * *code = 0 if no kernel reported an error.  Returns FE_EDEVICE if *code != 0. */
int fe_mesh_check_device(fe_mesh* mesh, void* stream, int32_t* code);

/* ------------------------------------------------------------------------
 * Column blocking (Alg. 2) and the closed block pattern (Sec. 3.5)
 * ------------------------------------------------------------------------ */

/* Alg. 2 for one process: locates the cell that contains each centre
 * (centres[3*n_cols], clamped into the box), sorts the columns by the position
 * of that cell in the ordered cell list of Alg. 1 (ties by column id), and
 * splits the sorted list into n_col_blocks contiguous groups whose sizes
 * differ by at most one (the first n_cols mod n_col_blocks groups are one
 * larger).  Outputs perm[n_cols] (new column j is old column perm[j]) and
 * col_block_ptr[n_col_blocks+1].  Widths must stay <= 16 (FE_EINVAL). */
int fe_column_blocks(const fe_mesh* mesh, int32_t n_cols, const double* centres,
                     int32_t n_col_blocks, int32_t* perm, int32_t* col_block_ptr);

/* Closed pattern of Sec. 3.5: given the support of each column block as a
 * set of DoF ids (supp_dofs[supp_ptr[c] .. supp_ptr[c+1]), any order,
 * duplicates allowed), block (r, c) is in the pattern iff row block r owns a
 * node of a cell that contains a support DoF of c.  Writes row_ptr
 * [n_row_blocks+1] and up to `capacity` column indices (ascending per row
 * block), and *nnz_blocks.  If capacity is too small nothing but *nnz_blocks
 * is written and FE_ENOMEM is returned, so a first call with capacity 0 sizes
 * the second. */
int fe_pattern_closed(const fe_mesh* mesh, int32_t n_col_blocks, const int64_t* supp_ptr,
                      const int64_t* supp_dofs, int64_t* row_ptr, int32_t* col_idx,
                      int64_t capacity, int64_t* nnz_blocks);

/* ------------------------------------------------------------------------
 * BCSR multivector (Sec. 3.3-3.4)
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t n_cols, n_col_blocks, n_row_blocks, dtype;
    int32_t max_width;            /* widest column block */
    int32_t pad_;
    int64_t nnz_blocks;           /* stored (row block, column block) blocks */
    int64_t n_values;             /* value slots, padding included */
    int64_t stored_entries;       /* sum over blocks of rows*width (padding excluded) */
    size_t value_bytes;           /* bytes of the value array */
    size_t table_bytes;           /* bytes of the device tables (tiles, Gram lists) */
    int64_t n_tiles;              /* (patch, column block) work items of the apply */
    int64_t active_cell_cols;     /* sum over tiles of active cells * width */
    int64_t n_gram_items_py;      /* work items of the P^T Y kernel */
    int64_t n_gram_items_pp;      /* work items of the P^T P kernel */
    double gram_flops;            /* sum_r sum_{c1,c2 in r} 2 rows_r w_c1 w_c2 (one product) */
} fe_bcsr_info_t;

/* Creates a BCSR multivector with n_cols columns split into column blocks
 * col_block_ptr[n_col_blocks+1] (widths 1..16) and the block pattern
 * row_ptr[n_row_blocks+1] / col_idx[nnz] (strictly ascending per row block,
 * in range; FE_EPATTERN otherwise).  dtype: FE_F32 or FE_F64.
 * Value layout: the blocks are stored one after another in CSR order; block
 * (r, c) holds rows_r rows (the DoFs of the row block in its local order) of
 * ld_c values each, row-major, where ld_c is the width w_c rounded up to a
 * multiple of 16 bytes (fe_bcsr_row_strides) so that every row starts on a
 * 16-byte boundary (the paper pads rows to a cache line, Sec. 3.5, for the
 * same reason: aligned vector access).  Entry (row, j) of the block, j < w_c,
 * is column col_block_ptr[c] + j.  Padding entries are ignored on input and
 * left zero on output.  Blocks start at the offsets of fe_bcsr_block_offsets. */
int fe_bcsr_create(const fe_mesh* mesh, int32_t n_cols, int32_t n_col_blocks,
                   const int32_t* col_block_ptr, const int64_t* row_ptr, const int32_t* col_idx,
                   int32_t dtype, fe_bcsr** out);
int fe_bcsr_destroy(fe_bcsr* bcsr);
int fe_bcsr_get_info(const fe_bcsr* bcsr, fe_bcsr_info_t* info);

/* offsets[nnz_blocks]: element offset of the first value of each block, in
 * CSR order. */
int fe_bcsr_block_offsets(const fe_bcsr* bcsr, int64_t* offsets);

/* ld[n_col_blocks]: row stride (elements) of the blocks of each column block. */
int fe_bcsr_row_strides(const fe_bcsr* bcsr, int32_t* ld);

/* Attaches the caller's device value array (value_bytes, 256-byte aligned)
 * and, when the multivector is used as the source P of fe_apply_H /
 * fe_gram_*, a device table buffer of table_bytes into which the tile and
 * Gram work lists are copied on `stream` (tables_dev may be NULL for a
 * destination Y).  Both pointers are kept until re-bound or destroyed. */
int fe_bcsr_bind(fe_bcsr* bcsr, void* values_dev, void* tables_dev, void* stream);
/* (values_dev may be NULL when the pattern is empty: value_bytes = 0.) */

/* ------------------------------------------------------------------------
 * Hot path (Alg. 6, Alg. 8)
 * ------------------------------------------------------------------------ */

/* Y = mask(P) * (H P): Alg. 6 with the destination restricted to P's block
 * pattern.  Runs the matrix-free cell operator (gather of the non-empty
 * column blocks of each patch, sum-factorised values and gradients at the
 * Gauss points, quadrature of 1/2 grad.grad + V, integration) and writes the
 * patch results into Y without atomics and without zeroing Y first: work
 * items are taken in descending patch rank, and each row of Y is stored by
 * the highest-ranked patch that contributes to it and then read, added to and
 * stored back by the others in descending rank, each waiting (on the GPU,
 * bounded in time) until its higher-ranked neighbour patches are done.  Every
 * stored entry of Y is overwritten, and the result is the same bit for bit
 * on every call.  The work counter and the per-patch completion counters live
 * in P's table buffer and are reset by each call, so two calls with the same
 * P (fe_apply_H, fe_apply_M, or the step calls) must not run concurrently.
 * P and Y must have identical patterns and dtype (FE_EPATTERN), P must be
 * bound with tables and Y with values (FE_ESTATE), the mesh uploaded and a
 * potential of the same dtype registered (FE_ESTATE).  A wait that gives up
 * sets the device status word (fe_mesh_check_device). */
int fe_apply_H(fe_mesh* mesh, const fe_bcsr* P, fe_bcsr* Y, void* stream);

/* Y = mask(P) * (M P) with the mass matrix M_ij = sum_K int_K N_i N_j
 * (Sec. 3.1, Eq. fe_matrices with the gradient term off and V = 1; Phi_M of
 * Sec. 2, whose Gram product P^T Y = P^T M P is the overlap matrix of
 * Eq. inner1).  Same kernels, layout, pattern rules and errors as
 * fe_apply_H, except that no potential needs to be registered.  Use
 * fe_gram_PtY(P, Y) for the overlap matrix. */
int fe_apply_M(fe_mesh* mesh, const fe_bcsr* P, fe_bcsr* Y, void* stream);

/* G = P^T Y (Alg. 8, Eq. inner2): dense n_cols x n_cols FP64, row-major, in
 * the column order of the multivectors, zero where no row block holds both
 * column blocks.  G_dev is caller-owned device memory (n_cols^2 doubles);
 * it is overwritten.  Accumulation is FP64 whatever the dtype.  Every block
 * of the product is formed, whatever Y holds. */
int fe_gram_PtY(const fe_bcsr* P, const fe_bcsr* Y, double* G_dev, void* stream);

/* The same product when the caller knows it to be symmetric: Y holds H P or
 * M P (fe_apply_H / fe_apply_M) of P's current values, and P's pattern is
 * closed for them (fe_bcsr_set_closed), so that mask(P) * (H P) = H P and
 * P^T Y = P^T H P (Eq. inner2; likewise P^T M P, Eq. inner1).  Only the
 * blocks c1 <= c2 are formed and mirrored, about half the work.  FE_ESTATE
 * if P is not declared closed.  For any other Y the result is wrong: use
 * fe_gram_PtY. */
int fe_gram_PtY_sym(const fe_bcsr* P, const fe_bcsr* Y, double* G_dev, void* stream);

/* G = P^T P (Alg. 8 / Eq. inner1 with the Euclidean product), same layout;
 * computed for column-block pairs c1 <= c2 and mirrored. */
int fe_gram_PtP(const fe_bcsr* P, double* G_dev, void* stream);

/* fe_apply_H then P^T Y on `stream`, and fe_gram_PtP (which does not
 * read Y) concurrently on a side stream owned by P, forked from `stream`
 * before the apply and joined back after P^T Y with events.  Y is formed
 * from P in the same call, so P^T Y takes the symmetric form of
 * fe_gram_PtY_sym when P is declared closed, else that of fe_gram_PtY.  All work
 * is ordered after earlier work on `stream` and before later work on it
 * (stream capture of the call records the fork and the join).  The side
 * stream is created on the first call and destroyed with P. */
int fe_apply_H_gram(fe_mesh* mesh, const fe_bcsr* P, fe_bcsr* Y, double* G_PY_dev,
                    double* G_PP_dev, void* stream);

/* End-to-end variant for callers whose data lives in host memory: copies
 * P's values from P_host (value_bytes) into P's bound device array, runs
 * the step of fe_apply_H_gram, copies Y's values to Y_host and both Gram
 * matrices to G_PY_host / G_PP_host, and synchronises `stream`.  The copies
 * overlap the kernels where the data allows: the apply runs as soon as P is
 * in, then Y leaves on a second stream owned by P (created on the first
 * call, destroyed with P) while P^T P (on P's side stream, G_PP leaving
 * after it) and P^T Y run.  On an error of the apply the call synchronises
 * `stream` and returns the apply's code; Y_host and the Gram buffers are
 * then not written.  Host buffers should be pinned for full copy bandwidth
 * and for the copies to run asynchronously. */
int fe_apply_H_gram_host(fe_mesh* mesh, const fe_bcsr* P, fe_bcsr* Y, double* G_PY_dev,
                         double* G_PP_dev, const void* P_host, void* Y_host,
                         double* G_PY_host, double* G_PP_host, void* stream);

/* Post-multiplication (Alg. 7, Sec. 3.6; Eqs. G_ops1/G_ops2):
 *   C = alpha (A X + gamma A) + beta C, truncated to C's block pattern,
 * where A and C have identical patterns and dtype (FE_EPATTERN otherwise) and
 * X_dev is an M x M FP64 matrix in device memory, row-major, in the
 * multivectors' column order.  The truncation of Alg. 7: products A_rk X_kj
 * whose column block j is not stored in row block r are discarded.  FP32
 * multivectors compute with X rounded to FP32 and FP32 FMAs (the result is
 * FP32); FP64 ones in FP64.  C's row padding is written as zero; A's row
 * padding must hold finite values (every routine here writes zeros there).
 * C must be bound with a table buffer: its pattern tables are used, and for
 * FP32 the rounded copy of X is written into it (so calls with the same C
 * must not overlap).  A needs values only.  C may not alias A (FE_EINVAL).  With gamma the orbital-minimisation gradient of Sec. 2,
 * G = -2 Phi_M Hbar + 2 Phi_H (2 I - Mbar), is
 *   fe_mmult(Phi_H, Mbar, -2, -2, 0, G);  fe_mmult(Phi_M, Hbar, -2, 0, 1, G).
 * FE_EUNSUPPORTED if the row strides of a row block's stored blocks add up
 * to more than 6144 columns. */
int fe_mmult(const fe_bcsr* A, const double* X_dev, double alpha, double gamma, double beta, fe_bcsr* C,
             void* stream);

/* Column-wise inner product tr(D^T G) = sum_alpha D_alpha . G_alpha over the
 * stored entries (Eq. G_ops4), for the line search.  D and G have identical
 * patterns and D is bound with a table buffer; the FP32 products are formed
 * and summed in FP64.  *out_dev (one double in device memory) is
 * overwritten. */
int fe_trace_dot(const fe_bcsr* D, const fe_bcsr* G, double* out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Launch configuration, CUDA graph of the step, autotuner.  These shape how
 * the kernels of Alg. 6 / Alg. 8 are launched on this GPU; the paper's method
 * is unchanged by them (Y is bit-identical under every launch shape; the Gram
 * products change only in the order of their FP64 additions).
 * ------------------------------------------------------------------------ */

/* Launch knobs of fe_apply_H for source multivector P:
 *   persistent      0: one CTA per work unit (grid launch); each CTA takes
 *                      its unit from the work counter in P's table buffer;
 *                   1: persistent launch of ctas_per_sm CTAs per SM that take
 *                      units from that counter until none is left;
 *   ctas_per_sm     1..32 (used by the persistent launch only);
 *   cells_per_round 0 = automatic, or 1, 2, 4, 8 = cap on the cells of the
 *                   patch a CTA holds at once (used by the p >= 3 kernel only).
 * Defaults: 0, 4, 0.  FE_EINVAL for values outside these ranges. */
int fe_bcsr_set_launch(fe_bcsr* P, int32_t persistent, int32_t ctas_per_sm, int32_t cells_per_round);

int fe_bcsr_get_launch(const fe_bcsr* P, int32_t* persistent, int32_t* ctas_per_sm,
                       int32_t* cells_per_round);

/* Caps the SMs that the persistent launches reading P may occupy: the
 * tensor-core Gram products (fe_gram_*, with P as A), the persistent apply
 * (fe_apply_H / fe_apply_M with P as source) and the tensor-core
 * post-multiplication (fe_mmult with P as A) launch at most max_sms SMs'
 * worth of CTAs.  0 (the default) = every SM.  Other streams' kernels then
 * find SMs free while these run (a server gives its large requests a cap and
 * its small ones the rest).  Results are unchanged.  FE_EINVAL for
 * max_sms < 0. */
int fe_bcsr_set_sm_limit(fe_bcsr* P, int32_t max_sms);

/* Declares (1) or withdraws (0, the default) that P's block pattern is closed
 * for the values P will hold: every row block that owns a node of a cell
 * touching the support of a column block is in that column block's pattern
 * (fe_pattern_closed builds such patterns, Sec. 3.5 reading).  Then
 * mask(P) * (H P) = H P, so P^T H P is symmetric: fe_apply_H_gram (and the
 * host-buffer variant and the graph of the step), which form Y = H P
 * themselves, compute its upper blocks only and mirror them, and
 * fe_gram_PtY_sym becomes available.  fe_gram_PtY is not affected.
 * Declaring it for a pattern that is not closed gives a wrong P^T Y in those
 * calls.  FE_EINVAL for a flag other than 0 or 1. */
int fe_bcsr_set_closed(fe_bcsr* P, int32_t closed);
int fe_bcsr_get_closed(const fe_bcsr* P, int32_t* closed);

/* Form of the cell operator that fe_apply_H and fe_apply_M use for source P.
 *   FE_FORM_SUMFAC  (default) sum factorisation, Alg. 6, on the FP32 or FP64
 *                   ALUs (every degree and dtype).
 *   FE_FORM_CELLMAT the element view H = sum_K P_K^T H_K P_K (Sec. 3.2, Eq.
 *                   fe_matrices_cell_based) with the element matrices applied
 *                   as dense products per cell, the approach the paper
 *                   compares against as "FE op. (BCSR gemm)" (Sec. 4.2).  On
 *                   the box mesh all cells share K_L (kinetic), S3 and Sb3, so
 *                   H_K u = K_L u + Sb3 (|J| V_K o S3 u) runs as two rounds of
 *                   TF32 tensor-core products with a 3-term split (FP32
 *                   accuracy); M_K u = (|J| Sb3 S3) u as one.  FE_F32 and
 *                   p <= 2 only.  Its launch is persistent (2 CTAs per SM) and
 *                   uses the work counter in P's tables, like the persistent
 *                   sum-factorised launch: two calls with the same P must not
 *                   run concurrently.
 * The result equals the other form's up to FP32 rounding (both within the
 * 1e-5 tolerance of the FP64 operator).  FE_EINVAL for another value,
 * FE_EUNSUPPORTED for FE_FORM_CELLMAT with FE_F64 values or p > 2. */
int fe_bcsr_set_form(fe_bcsr* P, int32_t form);
int fe_bcsr_get_form(const fe_bcsr* P, int32_t* form);

/* CUDA graph of one fe_apply_H_gram step with the given (already bound)
 * buffers: runs the step once eagerly on `stream` (this sets kernel
 * attributes and checks the arguments), then captures it on a private stream
 * and instantiates it.  The graph keeps the device pointers and launch
 * configuration of the moment of capture: re-create it after fe_bcsr_bind,
 * fe_mesh_set_potential or fe_bcsr_set_launch.  fe_graph_launch enqueues one
 * step on `stream`; fe_graph_destroy releases the graph (NULL is a no-op). */
typedef struct fe_graph fe_graph;
int fe_graph_create(fe_mesh* mesh, const fe_bcsr* P, fe_bcsr* Y, double* G_PY_dev, double* G_PP_dev,
                    void* stream, fe_graph** out);
int fe_graph_launch(fe_graph* graph, void* stream);
int fe_graph_destroy(fe_graph* graph);

/* Chooses the launch knobs of fe_apply_H for P by timing each candidate (five
 * calls after one warm-up, CUDA events on `stream`; Y is overwritten) and
 * sets the fastest with fe_bcsr_set_launch.  With a non-empty cache_path the
 * choice is looked up first (JSON lines, key = degree, dtype and work-list
 * sizes; the last matching line wins) and appended after a search.
 * *best_ms (may be NULL) receives the winner's time per call, or -1 on a
 * cache hit.  Candidates: p <= 2 grid launch and persistent with
 * 2..8 CTAs/SM; p >= 3 cells_per_round 8, 4, 2, 1. */
int fe_autotune(fe_mesh* mesh, fe_bcsr* P, fe_bcsr* Y, const char* cache_path, void* stream,
                double* best_ms);

/* ------------------------------------------------------------------------
 * Measurement helper (not part of the paper's method)
 * ------------------------------------------------------------------------ */

/* Runs an FMA-throughput probe on the current device (dtype FE_F32, FE_F64,
 * or 3 for packed FP32x2 FMA; eight independent chains per thread, 8 CTAs of
 * 256 threads per SM, `iters` x 128 FMAs per thread) and returns the achieved
 * flop/s (2 per FMA), the ALU peak used for the roofline of ALU-bound
 * kernels.  Thread 0 of every CTA stores its chain sum in the CTA's slot of
 * a sink; the call reads the first and last slot back and returns
 * FE_EDEVICE if they differ from the sum the host computes with the same
 * fused multiply-adds.  Synchronises `stream` (so it cannot be captured in
 * a CUDA graph); uses a small stream-ordered allocation for the sink. */
int fe_probe_fma(int32_t dtype, int64_t iters, double* flops_per_s, void* stream);

/* Allocation-free variant of fe_probe_fma (the paper has no counterpart: it
 * is a measurement helper).  Same arguments, kernels, check and result; the
 * per-CTA sink lives in a static device array of 4096 doubles (32 KB) that
 * every GPU which loads the library holds until the process exits, instead
 * of a stream-ordered allocation, so the call allocates no device memory at
 * all.  For callers that may not allocate, such as a server that has
 * admitted work up to its device-memory budget.
 *   - The first call on each device does a one-time set-up: with that
 *     device current it resolves the array's device address.  Like every
 *     call, it synchronises `stream`, so no call may be issued while a
 *     stream capture is in progress.
 *   - The slots are read back through the array's symbol, not through the
 *     resolved address, so a wrong address gives FE_EDEVICE.
 *   - FE_EINVAL with a message when the device needs more than 4096 slots
 *     (8 per SM, i.e. more than 512 SMs) or its ordinal is 64 or more.
 *   - All calls share the array, which keeps the last contents; nothing in
 *     it needs to start at zero (each CTA writes its own slot before the
 *     read-back).  Calls that overlap on the GPU (other streams or host
 *     threads) race on its contents and may fail the check. */
int fe_probe_fma_static(int32_t dtype, int64_t iters, double* flops_per_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FE_MF_H */
