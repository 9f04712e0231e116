// Internal declarations shared by the translation units of libfe.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>
#include <vector>

#include "fe.h"

namespace fe {

// ---------------------------------------------------------------- errors and streams
int set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
cudaStream_t cur_stream();
void count_launch();  // one of this library's kernels was launched

#define FE_CUDA(call)                                                      \
  do {                                                                     \
    cudaError_t _e = (call);                                               \
    if (_e != cudaSuccess) return fe::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)
#define FE_TRY(call)            \
  do {                          \
    int _rc = (call);           \
    if (_rc != FE_OK) return _rc; \
  } while (0)
#define FE_ARG(cond, ...)                                       \
  do {                                                          \
    if (!(cond)) return fe::set_error(FE_ERR_INVALID, __VA_ARGS__); \
  } while (0)

// Device buffer owned by RAII (cudaFree on destruction).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(size_t nbytes);         // FE_OK or FE_ERR_OOM; no-op when already large enough
  void release();
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline bool is_pow2_le16(int b) { return b == 1 || b == 2 || b == 4 || b == 8 || b == 16; }
// Block arguments are read and written with 16-byte vector accesses.
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
int num_sms();  // SMs of the current device

// Per-device launch set-up of one kernel, shared by every host thread.  The dynamic shared-
// memory limit is raised once on each device that launches the kernel; blocks per SM are cached
// per device and per launch shape (slot < kSetupSlots) and re-queried when a launch needs more
// shared memory than the cached figure was taken for.  One static KernelSetup per kernel.
constexpr int kMaxDevices = 64;
constexpr int kSetupSlots = 17;
struct KernelSetup {
  std::mutex mu;
  bool configured[kMaxDevices] = {};
  int per_sm[kMaxDevices][kSetupSlots] = {};
  size_t per_sm_smem[kMaxDevices][kSetupSlots] = {};
};
int cur_device();  // the current device's ordinal (FE_ERR_INVALID beyond kMaxDevices: < 0)
int kernel_configure(KernelSetup& ks, const void* func, int max_smem);
int kernel_occupancy(KernelSetup& ks, const void* func, int threads, size_t smem, int slot,
                     int* per_sm);

// ---------------------------------------------------------------- block descriptors
// A set of nv tall blocks; block j is n x bv with row stride ld (elements), starting at
// blk[j].  The eigensolver's subspace slots, a user's contiguous V and single columns of a
// block (bv = 1, ld = b) are all described this way.
constexpr int kMaxBlocks = 132;
// SpMM plan: rows of degree <= tail_max (at most kMaxTailDegree) go to degree-bucketed slices.
constexpr int kMaxTailDegree = 128;
constexpr int kDefaultTailMax = 128;
constexpr int kDefaultTailMaxPacked = 16;  // packed plans: most rows in the compressed tasks
constexpr int kMaxBuckets = kMaxTailDegree + 1;
// Rayleigh-Ritz: subspaces up to kRitzSmallMax are diagonalised entirely in shared memory by
// one CTA, up to 160 with the FP64 eigenvector matrix in a global workspace, and up to
// kRitzMax with FP32 sweeps on one CTA, FP64 products and cooperative FP64 sweeps on the grid.
constexpr int kRitzSmallMax = 96;
constexpr int kRitzMax = 512;
struct BlockSet {
  const void* blk[kMaxBlocks];
  int nv, bv, ld;
};
inline size_t dt_size(fe_dtype dt) { return dt == FE_F32 ? 4 : 8; }
// blk[j] = base + j * bstride elements
BlockSet make_blockset(const void* base, int nv, int bv, int ld, int64_t bstride, fe_dtype dt);
BlockSet blockset_of(const std::vector<const void*>& ptrs, int bv, int ld);

// G[(j*bv + p) * bw + q] = alpha * sum_r V_j[r][p] * W[r][q]  (FP64 out, device).
// Two phases (per-CTA partials, deterministic reduce); scratch from the gram scratch pool.
// engine (fe_engine): FP64 V and W go to the tensor-core kernel (tcgemm.cu) when it supports
// the shape (AUTO) or always (TC, error otherwise); FMA (default) keeps the FMA kernels.
int gram(const BlockSet& V, int64_t n, const void* W, int bw, int ldw, fe_dtype dt,
         double alpha, double* G, cudaStream_t s, int engine = FE_ENGINE_FMA);
// W[r] = beta * (W[r] M) + alpha * sum_j V_j[r] C_j   (M: bw x bw FP64 device or null = I;
// C: (nv*bv) x bw FP64 device; nv may be 0).
int update(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
           const double* M, void* W, int bw, int ldw, fe_dtype dt, cudaStream_t s);
// Out_o[r] = sum_j V_j[r] Y[j*bv.., o*bv..] for o < nout (Y: (nv*bv) x ldy FP64 device,
// output column block o uses Y columns [o*bv, (o+1)*bv)).  Out blocks must not alias V.
// engine (fe_engine): FP64 blocks go to the tensor-core split-product kernel (tcgemm.cu) when
// it supports the shape (AUTO) or always (TC, error otherwise); FMA keeps the FMA kernel.
int combine(const BlockSet& V, int64_t n, const double* Y, int ldy, const BlockSet& Out,
            fe_dtype dt, cudaStream_t s, int engine = FE_ENGINE_AUTO);
bool tc_combine_supported(const BlockSet& V, const BlockSet& Out, fe_dtype dt);
// Out = beta Out + alpha V Y (the beta term and the final sum in FP64; beta = 0: Out not read).
int tc_combine(const BlockSet& V, int64_t n, const double* Y, int ldy, const BlockSet& Out,
               cudaStream_t s, double alpha = 1.0, double beta = 0.0);
// G = alpha V^T W on the tensor cores (FP64 blocks; see tc_gram_supported for the shapes).
bool tc_gram_supported(const BlockSet& V, int bw, int ldw, fe_dtype dt);
int tc_gram(const BlockSet& V, int64_t n, const double* W, int bw, double alpha, double* G,
            cudaStream_t s);
// G[e] = alpha * sum over c < nctas of partial[c * nout + e], fixed order (deterministic).
int gram_reduce(const double* partial, int nctas, int nout, double alpha, double* G, cudaStream_t s);
// Small-matrix device scratch: a pool of FP64 buffers reused across calls on this thread.
double* small_scratch(int slot, size_t count);
int random_normal(void* X, int64_t n, int b, int ld, fe_dtype dt, uint64_t seed,
                  uint64_t stream, uint64_t offset, cudaStream_t s);
// dst[r][c] (dt) <- src (FP64, col-major with ld = n) or the transpose direction.
int convert_block(const void* src, fe_dtype sdt, int lds, void* dst, fe_dtype ddt, int ldd,
                  int64_t n, int b, cudaStream_t s);
int to_colmajor_f64(const BlockSet& X, int64_t n, int ncols, fe_dtype dt, double* out,
                    cudaStream_t s);

// Orthonormalise W (n x b, ld b) against V and itself; see fe_block_orth.  Synchronous.
struct OrthWork;
// vc32 (FP64, may be null): device flag; when set, V C is formed in FP32 arithmetic (for tiny
// correction coefficients only, see orth.cu).
int update_gram(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                const double* M, void* W, int b, fe_dtype dt, int gram_v, const int* skip,
                double* G, cudaStream_t s, const int* vc32 = nullptr);
int orth(const BlockSet& V, int64_t n, void* W, int b, fe_dtype dt, double* d_anorm,
         double anorm_floor, uint64_t seed, uint64_t* rng_counter, double* d_G, int ldg,
         double* d_R, int ldr, int* replaced, cudaStream_t s);

}  // namespace fe

// ---------------------------------------------------------------- the CSR handle
namespace fe {
struct SemiExt;
}
struct fe_spmm_plan {
  // tail: rows of degree 0..tail_max in 32-row slices grouped by degree (descending)
  int tail_max = 16;
  int64_t nslices = 0;
  int32_t* d_slice_rows = nullptr;   // nslices * 32 row ids (-1 = padding)
  int32_t* d_ell = nullptr;          // slice-major transposed column indices
  int32_t deg_slice_begin[fe::kMaxBuckets];  // first slice of degree d-bucket, in bucket order
  int64_t deg_ell_base[fe::kMaxBuckets];     // ELL offset of that bucket's first slice
  int32_t deg_of_bucket[fe::kMaxBuckets];
  int nbuckets = 0;
  // warp tasks: hub chunks first (partial slots 0..nhub_tasks-1), then mid rows by degree
  int64_t ntasks = 0, nhub_tasks = 0, nhub = 0;
  void* d_tasks = nullptr;           // struct Task[ntasks] (PTask when packed)
  uint32_t* d_tbits = nullptr;       // packed: the task rows' gap bit stream
  int packed = 0;
  int64_t index_bytes = 0;           // bytes of column-index data in the plan
  int32_t* d_hub_rows = nullptr;     // nhub
  int32_t* d_hub_task_begin = nullptr;  // nhub + 1
  int hub_min = 4096, hub_chunk = 4096;
  int l2_persist = 0;                // fe_csr_opts.l2_persist
};

struct fe_csr_s {
  int64_t n = 0, nnz = 0;
  int64_t ncols = 0;       // columns (= n except for a partition's rectangular row block)
  int device = 0;
  int64_t max_degree = 0;
  int64_t rows_empty = 0, rows_tail = 0, rows_mid = 0, rows_hub = 0;
  int32_t* d_colidx = nullptr;   // column indices of the warp-task rows (tail rows: in the ELL)
  fe_spmm_plan plan;
  fe::DevBuf partials;     // hub partial sums (nhub_tasks * 16 * 8 bytes)
  int64_t device_bytes = 0;
  // semi-external mode
  int semi_external = 0;
  fe::SemiExt* sx = nullptr;
  std::vector<void*> allocations;
  fe_csr_s* t = nullptr;   // A^T (fe_csr_opts.transpose), owned
};

namespace fe {
struct Task {
  int64_t start;  // offset into the plan's colidx
  int32_t row;    // output row
  int32_t len;    // non-zeros
};
// Warp task over bit-packed column gaps (index_format packed): the segment's sorted columns
// c_0 <= c_1 <= ... are stored as len fields of w bits, g_0 = 0 and g_k = c_k - c_{k-1},
// starting at word woff of the plan's bit stream (LSB first); c_k = base + g_0 + ... + g_k.
struct PTask {
  int64_t woff;
  int32_t row, len;
  int32_t base, w;
  int32_t pad0, pad1;
};
// Host-side SpMM plan of a row range (built at create; uploaded or packed into panels).
struct HostPlan {
  int64_t max_degree = 0, rows_empty = 0, rows_tail = 0, rows_mid = 0, rows_hub = 0;
  int nbuckets = 0;
  int32_t deg_of_bucket[kMaxBuckets], deg_slice_begin[kMaxBuckets];
  int64_t deg_ell_base[kMaxBuckets];
  int64_t nslices = 0, ell_total = 0, ntasks = 0, nhub_tasks = 0, nhub = 0, tcol_total = 0;
  std::vector<int32_t> slice_rows, ell, hub_rows, hub_task_begin;
  std::vector<int32_t> tcol;  // column indices of the task rows (mid and hub), in row order
  std::vector<Task> tasks;    // start: offset into tcol
  // packed index format: the task rows' columns as gap bit fields (tcol is then emptied)
  bool packed = false;
  std::vector<uint32_t> tbits;
  std::vector<PTask> ptasks;
};
// Device pointers of a plan (the resident handle's, or one streamed panel's).
struct PlanView {
  const int32_t* colidx;   // plain: task rows' column indices
  const uint32_t* tbits;   // packed: their gap bit stream (tasks are then PTask)
  int packed;
  const void* tasks;
  int64_t ntasks, nhub_tasks;
  const int32_t* slice_rows;
  const int32_t* ell;
  int64_t nslices;
  int nbuckets;
  int32_t deg_of_bucket[kMaxBuckets], deg_slice_begin[kMaxBuckets];
  int64_t deg_ell_base[kMaxBuckets];
  const int32_t* hub_rows;
  const int32_t* hub_task_begin;
  int64_t nhub;
  int64_t x_rows;          // rows of X (the matrix's columns), for the L2 window
  int l2_persist;          // 1: launch with an L2 access-policy window on X (persisting)
};
int build_host_plan(const int64_t* rowptr, const int32_t* colidx, int64_t r0, int64_t r1,
                    int tail_max, int hub_min, int hub_chunk, bool packed, HostPlan& hp);
// Bytes the column indices of row i take in a plan (ELL slice, plain task indices or packed
// gaps), for sizing panels.
size_t plan_row_index_bytes(const int32_t* cols, int64_t d, int tail_max, int hub_chunk, bool packed);
int spmm_view(const PlanView& v, const void* X, void* Y, void* partial, int b, fe_dtype dt,
              cudaStream_t s);
int spmm_resident(fe_csr h, const void* X, void* Y, int b, fe_dtype dt, cudaStream_t s);
int spmm_build_plan(fe_csr h, const int64_t* rowptr, const int32_t* colidx, int tail_max,
                    int hub_min, int hub_chunk, bool packed);
int semiext_create(fe_csr h, const int64_t* rowptr, const int32_t* colidx,
                   const fe_csr_opts& o);
int semiext_spmm(fe_csr h, const void* X, void* Y, int b, fe_dtype dt, cudaStream_t s);
void semiext_destroy(fe_csr h);
int64_t semiext_panels(fe_csr h);
}  // namespace fe
