/*
 * fe.h -- C ABI of the GB300-native FlashEigen hot path (arXiv 1602.01421).
 *
 * The paper's eigensolver (Section 3.1, Algorithm 1 with the block extension) builds a
 * subspace of m = b * NB vectors with sparse-matrix x dense-block multiplies (SpMM,
 * Section 3.3) and keeps it orthonormal with the dense tall-and-skinny operations of
 * Table 1 (MvTransMv, MvTimesMatAddMv, ...).  This library runs all of it on one GPU:
 *
 *   fe_csr_create / fe_csr_create_ex / fe_csr_destroy   the sparse matrix (Section 3.3.1)
 *   fe_spmm / fe_spmm_t                                  Y = A X, Y = A^T X (Section 3.3.3)
 *   fe_block_gram                                        MvTransMv  (Table 1, "op3")
 *   fe_block_update                                      MvTimesMatAddMv (Table 1, "op1")
 *   fe_block_update_gram                                 op1 then op3 on the result, one sweep
 *   fe_block_orth                                        re-orthogonalisation (Section 3.1)
 *   fe_random_normal                                     MvRandom (Table 1)
 *   fe_eigs / fe_eigs_ex                                 Block Krylov-Schur (Sections 1, 3.1)
 *   fe_svds                                              singular triplets via A^T A (4.3.2)
 *
 * Conventions shared by every entry point:
 *  - Return 0 (FE_OK) on success and a negative FE_ERR_* code on failure; fe_last_error()
 *    then returns a message for the calling thread.  No entry point aborts the process.
 *  - "device" pointers are CUDA device (or managed) memory of the current device; "host"
 *    pointers are ordinary host memory.  The caller owns every buffer it passes in.
 *  - Dense tall blocks are ROW-MAJOR n x b (element (r, c) at r*b + c), as the paper's SpMM
 *    wants its dense input (Section 3.3.2: row-major inside each row interval).  A set of
 *    nv blocks ("V") is stored block after block: block j starts at element j*n*b.  This is
 *    the paper's one-TAS-matrix-per-block subspace layout (Section 3.4.1) kept in HBM.
 *  - Small matrices (Gram results, coefficients) are FP64, row-major, in device memory.
 *  - Work is enqueued on the calling thread's current stream (fe_set_stream, default: the
 *    legacy default stream) and is asynchronous unless stated otherwise.
 *  - fe_dtype selects the element type of the tall blocks: FE_F32 = float, FE_F64 = double.
 */
#ifndef FE_H_
#define FE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FE_OK 0
#define FE_ERR_INVALID (-1)      /* bad argument or malformed CSR */
#define FE_ERR_OOM (-2)          /* device or pinned-host allocation failed */
#define FE_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define FE_ERR_NOCONVERGE (-4)   /* fe_eigs hit max_restarts; converged prefix returned */
#define FE_ERR_TIMEOUT (-5)      /* a bounded wait (semi-external copy) ran out */
#define FE_ERR_DEVICE_CHECK (-6) /* a kernel's own bounds/status check fired */

typedef struct fe_csr_s* fe_csr;

typedef enum { FE_F32 = 0, FE_F64 = 1 } fe_dtype;
typedef enum { FE_LM = 0, FE_LA = 1, FE_SA = 2 } fe_which; /* largest |x|, largest, smallest */
typedef enum { FE_MODE_FP64 = 0, FE_MODE_MIXED = 1 } fe_mode;
typedef enum { FE_START_RANDOM = 0, FE_START_USER = 1, FE_START_LEARNED = 2 } fe_start;
/* Arithmetic of the FP64 dense block products that support it (fe_block_combine and the
 * solver's restart and Ritz-vector products): FE_ENGINE_AUTO = tensor cores where the shape is
 * supported, FMA otherwise; FE_ENGINE_FMA = FP64 fused multiply-adds; FE_ENGINE_TC = tensor
 * cores (exact FP16 digit products, see fe_block_combine), FE_ERR_INVALID where unsupported. */
typedef enum { FE_ENGINE_AUTO = 0, FE_ENGINE_FMA = 1, FE_ENGINE_TC = 2 } fe_engine;

/* Message for the last failing call on this thread ("" if none).  Never NULL. */
const char* fe_last_error(void);

/* Library version string. */
const char* fe_version(void);

/* Number of this library's CUDA kernels launched by this process so far (all threads):
 * a diagnostic for benchmarks that report how many of their launches are the library's. */
int64_t fe_kernel_launches(void);

/* Set / get the CUDA stream (a cudaStream_t, NULL = legacy default stream) on which this
 * thread's subsequent calls enqueue work. */
int fe_set_stream(void* stream);
void* fe_get_stream(void);

/* ------------------------------------------------------------------ sparse matrix */

typedef enum { FE_INDEX_AUTO = 0, FE_INDEX_PLAIN = 1, FE_INDEX_PACKED = 2 } fe_index_format;

typedef struct {
  /* Cap, in bytes, on the device memory the CSR may occupy.  0 = no cap (the matrix is
   * resident in HBM).  When the resident layout would exceed it, the matrix stays in pinned
   * host memory and fe_spmm streams row panels through two device buffers: the paper's
   * semi-external SpMM (Section 3.3) with host memory in place of SSDs. */
  int64_t device_mem_cap_bytes;
  /* 1 = check that rowptr is monotone with rowptr[0] == 0 and every column index lies in
   * [0, n) (O(n + nnz) on the host).  Default 1.  0 skips the check, and the caller then
   * guarantees it: the SpMM kernels gather X rows at the stored indices without bounds checks. */
  int validate;
  /* 1 = additionally check that the pattern is symmetric and free of self-loops
   * (O(nnz log deg) on the host).  Default 0. */
  int check_symmetric;
  /* Rows with degree <= tail_max (at most 128) go to the degree-sorted slice format, one row
   * per lane (0 = default: 128; 16 for packed plans; semi-external handles with a small cap
   * may go lower to bound the slices' padding);
   * rows with degree > hub_min are split into chunks of hub_chunk non-zeros
   * (0 = defaults 4096 / 4096).  Tuning knobs only; results do not depend on them beyond
   * floating-point summation order. */
  int tail_max;
  int hub_min;
  int hub_chunk;
  /* Semi-external panel size in non-zeros (0 = default 64 Mi). */
  int64_t panel_nnz;
  /* Bound, in milliseconds, on each wait for a panel copy in semi-external mode (0 = 60000).
   * A wait that runs out makes fe_spmm return FE_ERR_TIMEOUT. */
  int copy_timeout_ms;
  /* Semi-external panel access: 0 = staged (each panel is copied into one of two device
   * buffers, copies overlapped with the previous panel's kernels); 1 = direct (the kernels read
   * the packed panels in pinned host memory through its device mapping, with no copies). */
  int semi_direct;
  /* Storage of the column indices of rows handled by warp tasks (degree > tail_max):
   * FE_INDEX_AUTO (0, default) = bit-packed gaps for semi-external handles, where the streamed
   * bytes bound the SpMM, plain int32 for resident ones; FE_INDEX_PLAIN = int32 indices;
   * FE_INDEX_PACKED = each row (each chunk of hub_chunk entries of a hub row) sorted and stored
   * as gaps to the previous column in fields of the row's largest gap width (the paper's
   * compressed-index idea, Section 3.3.1, in a GPU-decodable form: a warp reads 32 fields and
   * adds them up with a prefix sum).  Packed plans default to tail_max = 16. */
  int index_format;
  /* 1 = also build the transposed pattern A^T (host counting sort at create, then its own
   * SpMM plan), needed by fe_spmm_t and fe_svds: a directed graph's adjacency matrix is not
   * symmetric (Section 4.3.2).  With a device_mem_cap_bytes, A^T gets its own panels under the
   * same cap (the pair may hold up to twice the cap on the device).  Default 0. */
  int transpose;
  /* Columns of A (0 = n: square).  A rectangular n x ncols matrix -- one part's row block of a
   * row-partitioned matrix, with global column ids (fe_partition_local) -- must be resident,
   * without transpose or symmetry check; fe_spmm then reads ncols x b X and writes n x b Y, and
   * fe_eigs / fe_svds reject it. */
  int64_t ncols;
  /* 1 = launch the SpMM of a resident handle with an L2 access-policy window over X (persisting
   * hits, streaming misses, window up to the device's persisting set-aside, which the first such
   * launch on a device raises to its maximum for this process).  Default 0. */
  int l2_persist;
} fe_csr_opts;

/* Fill *opts with the defaults. */
void fe_csr_opts_default(fe_csr_opts* opts);

typedef struct {
  int64_t n, nnz;
  int64_t rows_empty;   /* degree 0 */
  int64_t rows_tail;    /* 1 <= degree <= tail_max */
  int64_t rows_mid;     /* tail_max < degree <= hub_min */
  int64_t rows_hub;     /* degree > hub_min */
  int64_t hub_chunks;   /* warp tasks the hub rows are split into */
  int64_t max_degree;
  int64_t device_bytes; /* device memory held by the handle */
  int semi_external;    /* 1 if the CSR streams from pinned host memory */
  int64_t panels;       /* semi-external row panels (0 when resident) */
  int has_transpose;    /* 1 if A^T was built (fe_csr_opts.transpose) */
  int tail_max;         /* the degree cutoff of the slice format in use (semi-external handles
                         * with the default may use a smaller one than resident ones) */
  int index_format;     /* FE_INDEX_PLAIN or FE_INDEX_PACKED, as in use */
  int64_t index_bytes;  /* bytes of column-index data in the plan (resident or streamed) */
  int64_t ncols;        /* columns (n unless created rectangular) */
} fe_csr_info;

/*
 * Create a handle for the n x n 0/1 sparse matrix A whose non-zeros in row i are the
 * columns colidx[rowptr[i] .. rowptr[i+1]-1] (CSR, Section 3.3.1; pattern only, every stored
 * entry is 1, as for the adjacency matrix of a graph).  rowptr (n+1 int64) and colidx
 * (nnz = rowptr[n] int32) are HOST pointers and are copied; the caller may free them when
 * the call returns.  n >= 1, 0 <= nnz.  Duplicate entries count twice (A_ij = multiplicity).
 * fe_eigs assumes A symmetric (the adjacency matrix of an undirected graph); fe_svds takes
 * any A (a directed graph) through A^T A.  Column indices need not be sorted within a row.
 * Errors: FE_ERR_INVALID (null pointers, n < 1, malformed rowptr, column out of range,
 * asymmetric pattern when check_symmetric, bad index_format), FE_ERR_OOM, FE_ERR_CUDA.
 * Synchronous.
 */
int fe_csr_create(int64_t n, const int64_t* rowptr, const int32_t* colidx, fe_csr* out);
int fe_csr_create_ex(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                     const fe_csr_opts* opts, fe_csr* out);
/* Release the handle and its device / pinned memory (synchronises the device first). */
int fe_csr_destroy(fe_csr h);
int fe_csr_get_info(fe_csr h, fe_csr_info* info);

/*
 * SpMM, Section 3.3.3: Y = A X, i.e. Y[i, :] = sum over the non-zeros (i, j) of X[j, :].
 * X and Y are DEVICE pointers to row-major ncols x b and n x b blocks of type dt, 1 <= b <= 16,
 * b in {1, 2, 4, 8, 16}; Y is overwritten (rows of empty matrix rows become 0); X and Y must
 * not overlap.  Accumulation is in dt.  Accuracy, per entry, against the exact sum of the
 * given X values, for any degree and any signs ((A|X|)_ij = sum over the row of |X[j, :]|):
 *   FP32: every lane's running sum is compensated (Kahan), lanes' sums are combined by a tree
 *         of at most 5 levels, and the chunks of a split hub row are added in compensated
 *         FP64 and rounded once, so |error| <= 9 * 2^-24 * (A|X|)_ij (about 5.4e-7, plus
 *         terms of order degree * 2^-48);
 *   FP64: plain sums, |error| <= (m + 6) * 2^-53 * (A|X|)_ij, m the longest run one lane adds:
 *         m <= tail_max for rows in the slices, m <= 512 for longer rows when X is 32-byte
 *         aligned (1024 when it is only 16-byte aligned and b = 16), so below 6e-14 (1.2e-13).
 * Both pointers must be 16-byte aligned.  Errors: FE_ERR_INVALID (null/unaligned pointer, unsupported b),
 * FE_ERR_CUDA, FE_ERR_TIMEOUT (semi-external copy wait).  Asynchronous when resident.
 */
int fe_spmm(fe_csr h, const void* X, void* Y, int b, fe_dtype dt);

/*
 * Transposed SpMM: Y = A^T X, i.e. Y[j, :] = sum over the non-zeros (i, j) of X[i, :] -- the
 * second half of the operator A^T A that the SVD of a directed graph's adjacency matrix
 * iterates with (Section 4.3.2).  Same arguments, layout and errors as fe_spmm; the handle
 * must have been created with fe_csr_opts.transpose = 1 (else FE_ERR_INVALID).  It runs the
 * fe_spmm kernels on the transposed pattern built at create.  Asynchronous.
 */
int fe_spmm_t(fe_csr h, const void* X, void* Y, int b, fe_dtype dt);

/* ------------------------------------------------------------------ block operations */
/* The n x b block arguments of the block operations below (V, W, Out) are read and written with
 * 16-byte vector accesses and must start on a 16-byte boundary (every cudaMalloc and torch
 * allocation does); an unaligned one gives FE_ERR_INVALID.  The small coefficient matrices
 * (C, Y, G, R) have no alignment requirement. */

/*
 * MvTransMv (Table 1, "op3"): G = alpha * V^T W.
 * V: DEVICE, nv blocks of n x bv (block j at element j*n*bv), so V^T W is (nv*bv) x bw.
 * W: DEVICE, n x bw row-major.  G: DEVICE, FP64 row-major (nv*bv) x bw, overwritten.
 * 1 <= nv <= 128, bv and bw in {1, 2, 4, 8, 16}; V and W may alias (W = one of V's blocks).
 * FP32 inputs: products and per-thread sums in FP32, cross-thread sums in FP64.  FP64 inputs:
 * tensor-core split products or FP64 FMA, as fe_block_gram_ex with FE_ENGINE_AUTO.
 * Errors: FE_ERR_INVALID, FE_ERR_OOM (scratch), FE_ERR_CUDA.
 */
int fe_block_gram(const void* V, int64_t n, int nv, int bv, const void* W, int bw,
                  fe_dtype dt, double alpha, double* G);

/*
 * fe_block_gram with a choice of arithmetic (fe_engine).  fe_block_gram is this call with
 * FE_ENGINE_AUTO.  For FP64 blocks with nv*bv <= 36 and bw in {1, 2, 4, 8}, FE_ENGINE_TC, and
 * FE_ENGINE_AUTO when nv*bv >= 16 (where it is the faster kernel), run on the tensor cores: within every 128-row tile each column of V and W is cut,
 * relative to its largest exponent in the tile, into seven 8-bit digits; one MMA per 16 rows
 * forms every digit product (exact FP16 x FP16 -> FP32 sums of 128 terms), and the tile's
 * products are assembled in integer arithmetic and added in FP64, so that the error of a tile's
 * contribution is at most 2^-50 * 128 * max|V[., c]| * max|W[., q]| over its rows (plus the
 * FP64 roundings of the sums over tiles); entries must be finite, subnormals are read as zero.
 * Otherwise, and with FE_ENGINE_FMA, the FMA kernels of fe_block_gram.  FE_ENGINE_TC with an
 * unsupported shape or FP32 blocks: FE_ERR_INVALID.
 */
int fe_block_gram_ex(const void* V, int64_t n, int nv, int bv, const void* W, int bw,
                     fe_dtype dt, double alpha, double* G, int engine);

/*
 * fe_block_gram without any device allocation.  The paper has no counterpart; this entry point
 * exists for callers that cannot let the library call cudaMalloc: programs whose device
 * memory is reserved up front by their own allocator, with nothing left to hand out, and code
 * that must not make calls that can synchronise the whole device, as cudaMalloc and cudaFree
 * may.  Arguments, layouts, result and error codes are those of fe_block_gram, except:
 *  - nv * bv * bw must be at most 2048 (larger G: FE_ERR_INVALID with a message);
 *  - the per-CTA partial sums live in a 2 MiB static device array inside the library, which
 *    every GPU that loads the library holds until the process exits;
 *  - the first call on each device looks up that array's device address (done with the
 *    device current, kept for later calls); make that first call before any stream capture;
 *  - all calls share the array, so calls whose work overlaps on the GPU (other streams, other
 *    host threads) race; each call writes every partial it reads, so nothing needs clearing.
 */
int fe_block_gram_noalloc(const void* V, int64_t n, int nv, int bv, const void* W, int bw,
                          fe_dtype dt, double alpha, double* G);

/*
 * MvTimesMatAddMv (Table 1, "op1"): W = beta * W + alpha * V C.
 * V: DEVICE, nv blocks of n x bv; C: DEVICE FP64 row-major (nv*bv) x bw; W: DEVICE n x bw.
 * nv = 0 gives MvScale1 (W = beta W).  W must not alias V.  1 <= nv <= 128 (or 0),
 * bv, bw in {1, 2, 4, 8, 16}.  Errors: FE_ERR_INVALID, FE_ERR_CUDA.
 */
int fe_block_update(const void* V, int64_t n, int nv, int bv, const double* C, double alpha,
                    double beta, void* W, int bw, fe_dtype dt);

/*
 * fe_block_update with a choice of arithmetic (fe_engine); fe_block_update is this call with
 * FE_ENGINE_FMA.  For FP64 with nv >= 1, bv == bw, K = nv*bv <= 64 and bw <= 32,
 * FE_ENGINE_AUTO and FE_ENGINE_TC form alpha V C on the tensor cores as fe_block_combine does
 * (split products, the same error bound, with alpha folded into C before it is split) and add
 * it to beta W in FP64 (one rounding); the update of the second Gram-Schmidt pass, W - V G1.
 * Otherwise, and for FE_ENGINE_FMA, FMA kernels in dt.  Errors: as fe_block_update, and
 * FE_ERR_INVALID for FE_ENGINE_TC with an unsupported shape or dtype.  Asynchronous.
 */
int fe_block_update_ex(const void* V, int64_t n, int nv, int bv, const double* C, double alpha,
                       double beta, void* W, int bw, fe_dtype dt, int engine);

/*
 * MvTimesMatAddMv followed by MvTransMv on its result (Table 1 "op1" then "op3"), the pair the
 * second classical Gram-Schmidt pass of Section 3.1 issues, fused into one sweep over the rows:
 *     W <- beta * W + alpha * V C,      G = [V_0; ...; V_{nv-1}; W]^T W   (W after the update)
 * V: DEVICE, nv blocks of n x b (block after block); C: DEVICE FP64 row-major (nv*b) x b;
 * W: DEVICE n x b, updated in place; G: DEVICE FP64 row-major ((nv+1)*b) x b, rows j*b + p
 * for block j's column p, then W's b rows.  0 <= nv <= 128 (nv = 0: W = beta W, G = W^T W),
 * b in {1, 2, 4, 8}.  W must not alias V.  Deterministic (fixed summation order).
 * Errors: FE_ERR_INVALID, FE_ERR_OOM, FE_ERR_CUDA.
 */
int fe_block_update_gram(const void* V, int64_t n, int nv, int b, const double* C, double alpha,
                         double beta, void* W, fe_dtype dt, double* G);

/*
 * Block product with several output blocks, the restart and Ritz-vector product of the
 * Krylov-Schur solver, V_new = V Y (Table 1 "op1", MvTimesMatAddMv with beta = 0; Section 3.1
 * step (2)): output block o (n x bv) = sum_j V_j Y[j*bv:(j+1)*bv, o*bv:(o+1)*bv].
 * V: DEVICE, nv blocks of n x bv (block after block); Y: DEVICE FP64 row-major
 * (nv*bv) x (nout*bv); Out: DEVICE, nout blocks of n x bv, overwritten, must not alias V.
 * 1 <= nv <= 128, 1 <= nout <= 128, bv in {1, 2, 4, 8, 16}.
 * engine (fe_engine): for FP64 with K = nv*bv <= 64 and N = nout*bv <= 32, FE_ENGINE_AUTO and
 * FE_ENGINE_TC use the tensor cores: every V row is cut, relative to its largest exponent, into
 * seven 8-bit digits, every Y column likewise; the digit products (exact in FP16 x FP16 -> FP32
 * for K <= 32 per accumulator) of weight classes i + j <= 6 are summed on the tensor cores,
 * assembled in integer arithmetic (two 64-bit words, then the value without its 12 lowest bits)
 * and rounded once, so that |error| <= 2^-49 (K + 1) max_c|V[r][c]| max_c|Y[c][q]|
 * + 2^-52 |result| (results below 2^-1022 flush to zero; entries must be finite,
 * subnormal entries are read as zero).  Otherwise, and for FE_ENGINE_FMA, FMA kernels in dt
 * (FP32 blocks: FP32 arithmetic).  Errors: FE_ERR_INVALID (including FE_ENGINE_TC with an
 * unsupported shape), FE_ERR_OOM, FE_ERR_CUDA.  Asynchronous.
 */
int fe_block_combine(const void* V, int64_t n, int nv, int bv, const double* Y, int nout, void* Out,
                     fe_dtype dt, int engine);

/*
 * Re-orthogonalisation step of the block Krylov expansion (Section 3.1 step (1)): block
 * classical Gram-Schmidt run twice against the orthonormal basis V (nv blocks of n x b,
 * DEVICE), then CholeskyQR2 of the remainder, so that on return
 *     W_in = V G + W_out R,  W_out^T W_out = I,  V^T W_out = 0.
 * W (DEVICE, n x b) is overwritten by W_out.  G (DEVICE FP64 (nv*b) x b) and R (DEVICE FP64
 * b x b, upper triangular) receive the coefficients.  nv may be 0 (plain CholeskyQR2).
 * anorm is the scale of ||A|| used by the breakdown test: a column whose remainder falls
 * below 1e-12 * anorm is replaced by a random direction (seed, counter stream 5) orthogonal
 * to V and the earlier columns, with R[i][i] = 0.  *replaced (HOST, may be NULL) receives the
 * number of replaced columns.  Synchronous.  Errors: FE_ERR_INVALID, FE_ERR_OOM, FE_ERR_CUDA.
 */
int fe_block_orth(const void* V, int64_t n, int nv, int b, void* W, fe_dtype dt,
                  double anorm, uint64_t seed, double* G, double* R, int* replaced);

/*
 * MvRandom (Table 1): fill the DEVICE row-major n x b block X with N(0, 1) draws from the
 * counter-based generator: element (r, c) has index i = offset + r*b + c and takes
 * u1, u2 = the top 53 bits of SplitMix64(seed, stream, 2i), (.., 2i+1) scaled to [0, 1),
 * z = sqrt(-2 ln(1 - u1)) cos(2 pi u2)  (Box-Muller).  Errors: FE_ERR_INVALID, FE_ERR_CUDA.
 */
int fe_random_normal(void* X, int64_t n, int b, fe_dtype dt, uint64_t seed, uint64_t stream,
                     uint64_t offset);

/* ------------------------------------------------------------------ row partition (multi-GPU) */
/* The paper's solver runs on one machine (Section 3); across several GPUs the method shards by
 * rows: a part owns a contiguous row range of A and of every n x b block, an SpMM needs the X
 * rows its column indices reference (an all-gather of X, or only the "halo" rows), and a Gram
 * product V^T W is the sum of the parts' partial products (an all-reduce of the small result).
 * These host functions compute the partition and a part's local CSR; the exchanges are the
 * caller's (the Python package's dist module over torch.distributed). */

/* Split rows [0, n) of the CSR into nparts contiguous ranges of near-equal cost (non-zeros +
 * rows): part p owns rows [row_begin[p], row_begin[p+1]).  rowptr: HOST, n+1 entries;
 * row_begin: HOST, nparts+1 entries, written.  Each part's cost is at most total/nparts plus
 * the cost of one row.  Errors: FE_ERR_INVALID (NULL, n < 1, nparts < 1, decreasing rowptr). */
int fe_partition_rows(int64_t n, const int64_t* rowptr, int nparts, int64_t* row_begin);

/* The local CSR of rows [r0, r1): local_rowptr (HOST, r1-r0+1 entries, starting at 0) and
 * local_colidx (HOST, rowptr[r1]-rowptr[r0] entries) keep GLOBAL column ids in the original
 * order; halo (HOST, may be NULL; room for rowptr[r1]-rowptr[r0] entries) receives the sorted
 * distinct columns outside [r0, r1), *nhalo their number.  Errors: FE_ERR_INVALID. */
int fe_partition_local(int64_t n, const int64_t* rowptr, const int32_t* colidx, int64_t r0, int64_t r1,
                       int64_t* local_rowptr, int32_t* local_colidx, int32_t* halo, int64_t* nhalo);

/* ------------------------------------------------------------------ learned start block */
/* Not in the paper (its solver starts from MvRandom, Table 1): a small MLP maps per-vertex
 * features computed with SpMM (Section 3.3) to an n x b start block.  Features, network and
 * loss are specified in the comments of fe_vertex_features / fe_mlp_forward /
 * fe_mlp_loss_grad; all arrays are DEVICE, row-major, FP32 unless stated. */
#define FE_NFEAT 8

/* Number of packed MLP parameters for hidden width `hidden` (32 or 64) and b outputs
 * (1, 2, 4, 8, 16): 8H + H + H^2 + H + Hb + b, packed as [W1 (8 x H), b1, W2 (H x H), b2,
 * W3 (H x b), b3], row-major.  Returns -1 for unsupported sizes. */
int64_t fe_mlp_param_count(int hidden, int b);

/* F (n x 8): d = A 1; f0 = log(1+d), f1 = d/rms(d), f2 = A d/rms(A d), f3 = A^2 d/rms(A^2 d);
 * with R = N(0,1) n x 4 from the counter generator (seed, stream 6) and q_p = mean over
 * columns of (A^p R)^2 (p = 2, 3, 4): f4 = q2/rms(q2), f5 = q3/rms(q3), f6 = q4/rms(q4),
 * f7 = log(1 + q2/mean(q2)); rms(x) = sqrt(mean(x^2)) (1 if 0).  SpMMs in FP64, F in FP32.
 * Synchronous.  Errors: FE_ERR_INVALID, FE_ERR_OOM, FE_ERR_CUDA. */
int fe_vertex_features(fe_csr h, uint64_t seed, float* F);

/* Z (n x b) = relu(relu(F W1 + b1) W2 + b2) W3 + b3. */
int fe_mlp_forward(const float* F, int64_t n, const float* params, int hidden, int b, float* Z);

/* Loss L = sum_j (1 - (z_j . u_j)^2 / |z_j|^2) of the network output Z against U (n x b, unit
 * columns; invariant to each column's sign) and its gradient with respect to the packed
 * parameters (grad: DEVICE, fe_mlp_param_count floats, overwritten).  loss: HOST, may be NULL
 * (when given the call synchronises).  Sums over rows are per-CTA partials added in order in
 * FP64 (deterministic). */
int fe_mlp_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                     const float* U, float* grad, double* loss);

/* Subspace form of the loss, invariant to any rotation of the targets: U (n x t) is an
 * orthonormal target basis (e.g. the nev wanted Ritz vectors) and
 * L = sum_j (1 - |U^T z_j|^2 / |z_j|^2), the part of each output column outside span(U).
 * hidden = 64, b in {4, 8}, t in {4, 8, 16}.  Otherwise as fe_mlp_loss_grad. */
int fe_mlp_subspace_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                              const float* U, int t, float* grad, double* loss);

/* Span form, invariant to rotations of U and to any invertible mixing of the outputs:
 * L = b - tr((Z^T Z)^{-1} Z^T U U^T Z), b minus the squared cosines of the principal angles
 * between span(Z) and span(U), so b copies of one good direction score as one.  hidden = 64,
 * (b, t) in {(4, 4), (4, 8), (8, 8)}.  Otherwise as fe_mlp_loss_grad. */
int fe_mlp_span_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                          const float* U, int t, float* grad, double* loss);

/* One Adam step (Kingma & Ba 2015, bias-corrected; step counts from 1) on count parameters. */
int fe_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count, double lr,
                double beta1, double beta2, double eps, int step);

/* ------------------------------------------------------------------ eigensolver */

typedef struct {
  uint64_t seed;          /* counter-RNG seed for the random start / replacements (1) */
  int max_restarts;       /* restart cycles before FE_ERR_NOCONVERGE (500) */
  fe_mode mode;           /* FE_MODE_FP64 or FE_MODE_MIXED (FP32 subspace + FP64 refine) */
  fe_start start;         /* FE_START_RANDOM, FE_START_USER (start_block) or _LEARNED */
  const void* start_block;/* DEVICE row-major n x block FP64, for FE_START_USER */
  const float* mlp_weights; /* DEVICE packed MLP parameters (fe_mlp_param_count floats,
                             b = block), for FE_START_LEARNED; features use `seed` */
  int mlp_hidden;         /* hidden width of that MLP: 32 or 64 (64) */
  double mixed_tol;       /* FP32-phase tolerance in mixed mode (5e-6) */
  int max_sweeps;         /* Jacobi sweeps per Rayleigh-Ritz (60) */
  int orth_pass1;         /* FP64 subspace, first Gram-Schmidt pass: 0 = its Gram in FP32
                             arithmetic (the FP64 second pass restores full orthogonality, and
                             the coefficients actually subtracted enter H, so the Krylov
                             relation keeps FP64 accuracy), 1 = in FP64 (0) */
  int subspace_host;      /* 1 = keep the subspace blocks in pinned host memory that the GPU
                             reads and writes over the CPU-GPU link (the paper's external-memory
                             vector subspace, Section 3.4.3), with the newest block cached in
                             device memory for the next SpMM (its most-recent-matrix caching,
                             Section 3.4.4); for subspaces larger than HBM.  Same arithmetic,
                             same results as 0 (default). */
  int engine;             /* FP64 restart and Ritz-vector products: FE_ENGINE_FMA = FP64 FMA,
                             FE_ENGINE_AUTO or FE_ENGINE_TC = tensor cores wherever
                             fe_block_combine supports the shape (subspace m <= 64, kept
                             vectors <= 32), and the second Gram-Schmidt pass (update and
                             Gram) on the tensor cores where the shapes allow (nv*b <= 36,
                             b <= 8); FP64 FMA elsewhere (FE_ENGINE_AUTO) */
  int orth_local;         /* FP64 subspace, first Gram-Schmidt pass of a new block W = A v_j:
                             1 = its coefficients against the older blocks v_i (i < j) are read
                             from the projected matrix, v_i^T A v_j = H[j][i] for symmetric A
                             (the Lanczos recurrence: nonzero only for v_{j-1} and, after a
                             restart, the kept vectors), and only v_j^T W is computed; the
                             second pass is the full Gram as always (1); 0 = a full Gram in the
                             first pass too.  FP32 subspaces (the mixed mode's first phase)
                             always take the full first pass: there it keeps the restart
                             count lower */
} fe_eigs_opts;

void fe_eigs_opts_default(fe_eigs_opts* opts);

typedef struct {
  int nconv;              /* wanted pairs that passed the convergence test */
  int restarts;           /* restart cycles run (all phases) */
  int64_t spmm_blocks;    /* n x b block SpMMs (all phases) */
  int64_t spmm_blocks_fp32; /* of which in the FP32 phase (mixed mode) */
  int restarts_fp32;      /* restart cycles of the FP32 phase (mixed mode) */
  int replacements;       /* breakdown columns replaced by random directions */
  double anorm;           /* final estimate of ||A||_2 (largest |theta| seen) */
  double max_resid;       /* max explicit ||A x - theta x|| over the returned pairs */
  double seconds;         /* wall time of the call */
  double seconds_fp32;    /* of which in the FP32 phase (mixed mode) */
  int64_t spmm_start;     /* SpMM calls spent building the start block (learned start: 7) */
} fe_eigs_stats;

/*
 * Block Krylov-Schur eigensolver (Sections 1 and 3.1): the nev eigenpairs of the symmetric
 * 0/1 matrix of h that come first in `which` order (FE_LM: |lambda| descending, ties ->
 * larger lambda first; FE_LA: descending; FE_SA: ascending).  block = b, nblocks = NB,
 * subspace m = b * NB; requires 1 <= nev <= m - b, m + b <= n, b in {1, 2, 4, 8, 16},
 * NB >= 2, m <= 512, NB <= 130 (m > 96: the projected eigenproblem keeps its matrices in a device
 * workspace that fe_eigs allocates, 2 (m+1)^2 doubles up to m = 160 and 5 (m+1)^2 above; above
 * m = 160 it runs FP32 Jacobi sweeps on one CTA, FP64 matrix products and FP64 Jacobi sweeps on a
 * cooperative grid).  A pair is converged when its Ritz residual estimate is at most
 * tol * max(|theta|, 1e-3 * max|theta|) and the explicit residual ||A x - theta x|| passes the
 * same test.  evals: HOST, nev doubles.  evecs: DEVICE, n x nev COLUMN-major FP64 (ConvLayout,
 * Table 1), may be NULL; each vector's largest-magnitude entry is positive.  Synchronous.
 * Returns FE_ERR_NOCONVERGE after max_restarts with the converged count in stats->nconv and
 * the current Ritz pairs in evals/evecs.
 */
int fe_eigs(fe_csr h, int nev, int block, int nblocks, double tol, fe_which which,
            double* evals, double* evecs);
int fe_eigs_ex(fe_csr h, int nev, int block, int nblocks, double tol, fe_which which,
               const fe_eigs_opts* opts, double* evals, double* evecs, fe_eigs_stats* stats);

/*
 * Singular value decomposition of a (directed graph's) 0/1 matrix A, Section 4.3.2: the nsv
 * largest singular values sigma_1 >= ... >= sigma_nsv with right and left singular vectors.
 * The Block Krylov-Schur iteration of fe_eigs_ex runs on the symmetric positive semidefinite
 * operator A^T A (one fe_spmm and one fe_spmm_t per block), largest eigenvalues first; then
 * sigma_i = sqrt(theta_i), v_i = the Ritz vectors, u_i = A v_i / sigma_i (0 if sigma_i = 0).
 * The convergence test is fe_eigs_ex's, applied to A^T A (tol relative to theta = sigma^2).
 * The handle needs fe_csr_opts.transpose = 1 (resident or semi-external).  block, nblocks, opts as
 * for fe_eigs_ex (modes FP64 and MIXED; starts RANDOM and USER; FE_START_LEARNED is rejected).
 * svals: HOST, nsv doubles.  right, left: DEVICE, n x nsv COLUMN-major FP64, each may be
 * NULL; each v_i has its largest-magnitude entry positive.  stats->spmm_blocks counts
 * applications of A^T A (two SpMMs each).  Synchronous.  Errors as fe_eigs_ex.
 */
int fe_svds(fe_csr h, int nsv, int block, int nblocks, double tol, const fe_eigs_opts* opts,
            double* svals, double* right, double* left, fe_eigs_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* FE_H_ */
