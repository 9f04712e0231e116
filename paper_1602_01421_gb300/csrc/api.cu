// C-ABI entry points: errors, streams, the CSR handle and the Table 1 block operations.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

static thread_local char g_err[1024] = "";
static thread_local cudaStream_t g_stream = nullptr;

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  int code = (e == cudaErrorMemoryAllocation) ? FE_ERR_OOM : FE_ERR_CUDA;
  set_error(code, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return code;
}

cudaStream_t cur_stream() { return g_stream; }

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int DevBuf::alloc(size_t nbytes) {
  if (nbytes <= bytes && p) return FE_OK;
  release();
  if (nbytes == 0) return FE_OK;
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    cudaGetLastError();
    return set_error(FE_ERR_OOM, "cudaMalloc(%zu) failed: %s", nbytes, cudaGetErrorString(e));
  }
  bytes = nbytes;
  return FE_OK;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

int num_sms() {
  static std::atomic<int> sms[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices) dev = 0;
  int v = sms[dev].load(std::memory_order_relaxed);
  if (!v) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    v = v > 0 ? v : 1;
    sms[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

int cur_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(FE_ERR_INVALID, "device ordinal %d beyond the library's %d", dev, kMaxDevices);
  return dev;
}

int kernel_configure(KernelSetup& ks, const void* func, int max_smem) {
  const int dev = cur_device();
  if (dev < 0) return dev;
  std::lock_guard<std::mutex> lock(ks.mu);
  if (!ks.configured[dev]) {
    FE_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    ks.configured[dev] = true;
  }
  return FE_OK;
}

int kernel_occupancy(KernelSetup& ks, const void* func, int threads, size_t smem, int slot,
                     int* per_sm) {
  const int dev = cur_device();
  if (dev < 0) return dev;
  FE_ARG(slot >= 0 && slot < kSetupSlots, "internal: launch-shape slot %d", slot);
  std::lock_guard<std::mutex> lock(ks.mu);
  if (ks.per_sm[dev][slot] == 0 || smem > ks.per_sm_smem[dev][slot]) {
    int nb = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, smem));
    ks.per_sm[dev][slot] = std::max(nb, 1);
    ks.per_sm_smem[dev][slot] = smem;
  }
  *per_sm = ks.per_sm[dev][slot];
  return FE_OK;
}

BlockSet make_blockset(const void* base, int nv, int bv, int ld, int64_t bstride, fe_dtype dt) {
  BlockSet s;
  memset(&s, 0, sizeof(s));
  s.nv = nv;
  s.bv = bv;
  s.ld = ld;
  for (int j = 0; j < nv && j < kMaxBlocks; ++j)
    s.blk[j] = base ? (const char*)base + (size_t)j * bstride * dt_size(dt) : nullptr;
  return s;
}

BlockSet blockset_of(const std::vector<const void*>& ptrs, int bv, int ld) {
  BlockSet s;
  memset(&s, 0, sizeof(s));
  s.nv = (int)ptrs.size();
  s.bv = bv;
  s.ld = ld;
  for (int j = 0; j < s.nv && j < kMaxBlocks; ++j) s.blk[j] = ptrs[j];
  return s;
}

}  // namespace fe

using namespace fe;

extern "C" {

const char* fe_last_error(void) { return g_err; }
const char* fe_version(void) { return "fe-gb300 0.1 (sm_103a)"; }
int64_t fe_kernel_launches(void) { return g_launches.load(); }

int fe_set_stream(void* stream) {
  g_stream = reinterpret_cast<cudaStream_t>(stream);
  return FE_OK;
}
void* fe_get_stream(void) { return reinterpret_cast<void*>(g_stream); }

void fe_csr_opts_default(fe_csr_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->validate = 1;
}

static int validate_csr(int64_t n, int64_t ncols, const int64_t* rowptr, const int32_t* colidx) {
  if (rowptr[0] != 0) return set_error(FE_ERR_INVALID, "rowptr[0] = %lld, expected 0", (long long)rowptr[0]);
  int64_t bad_row = -1;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) { bad_row = i; break; }
  if (bad_row >= 0) return set_error(FE_ERR_INVALID, "rowptr decreases at row %lld", (long long)bad_row);
  int64_t nnz = rowptr[n];
  int64_t bad = -1;
  #pragma omp parallel for schedule(static) reduction(max : bad)
  for (int64_t p = 0; p < nnz; ++p)
    if (colidx[p] < 0 || colidx[p] >= ncols) bad = std::max(bad, p);
  if (bad >= 0)
    return set_error(FE_ERR_INVALID, "colidx[%lld] = %d out of range [0, %lld)", (long long)bad,
                     colidx[bad], (long long)ncols);
  return FE_OK;
}

// Pattern of A^T: the non-zero (i, j) becomes (j, i).  Counting sort by column; rows of A are
// visited in order, so every row of A^T comes out sorted.
static void transpose_pattern(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                              std::vector<int64_t>& trp, std::vector<int32_t>& tci) {
  const int64_t nnz = rowptr[n];
  trp.assign(n + 1, 0);
  for (int64_t p = 0; p < nnz; ++p) trp[colidx[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) trp[i + 1] += trp[i];
  tci.resize(nnz > 0 ? nnz : 1);
  std::vector<int64_t> cur(trp.begin(), trp.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) tci[cur[colidx[p]]++] = (int32_t)i;
}

static int check_symmetric(int64_t n, const int64_t* rowptr, const int32_t* colidx) {
  // transpose by counting sort, then compare the sorted rows of A and A^T
  int64_t nnz = rowptr[n];
  std::vector<int64_t> tp(n + 1, 0);
  for (int64_t p = 0; p < nnz; ++p) tp[colidx[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) tp[i + 1] += tp[i];
  std::vector<int32_t> tc(nnz);
  std::vector<int64_t> cur(tp.begin(), tp.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (colidx[p] == i) return set_error(FE_ERR_INVALID, "self-loop at row %lld", (long long)i);
      tc[cur[colidx[p]]++] = (int32_t)i;
    }
  int64_t bad = -1;
  #pragma omp parallel for schedule(dynamic, 1024) reduction(max : bad)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<int32_t> a(colidx + rowptr[i], colidx + rowptr[i + 1]);
    std::sort(a.begin(), a.end());
    // tc rows are already sorted (rows visited in order)
    if (!std::equal(a.begin(), a.end(), tc.begin() + tp[i], tc.begin() + tp[i + 1]) ||
        (int64_t)a.size() != tp[i + 1] - tp[i])
      bad = std::max(bad, i);
  }
  if (bad >= 0) return set_error(FE_ERR_INVALID, "pattern is not symmetric (row %lld)", (long long)bad);
  return FE_OK;
}

int fe_csr_create(int64_t n, const int64_t* rowptr, const int32_t* colidx, fe_csr* out) {
  fe_csr_opts o;
  fe_csr_opts_default(&o);
  return fe_csr_create_ex(n, rowptr, colidx, &o, out);
}

int fe_csr_destroy(fe_csr h) {
  if (!h) return FE_OK;
  cudaDeviceSynchronize();
  if (h->t) fe_csr_destroy(h->t);
  if (h->semi_external) semiext_destroy(h);
  for (void* p : h->allocations) cudaFree(p);
  delete h;
  return FE_OK;
}

int fe_csr_create_ex(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                     const fe_csr_opts* opts, fe_csr* out) {
  FE_ARG(out != nullptr, "fe_csr_create: out is NULL");
  *out = nullptr;
  FE_ARG(n >= 1 && n <= INT32_MAX, "fe_csr_create: n = %lld must be in [1, 2^31)", (long long)n);
  FE_ARG(rowptr != nullptr, "fe_csr_create: rowptr is NULL");
  fe_csr_opts o;
  fe_csr_opts_default(&o);
  if (opts) o = *opts;
  int64_t nnz = rowptr[n];
  FE_ARG(nnz >= 0, "fe_csr_create: rowptr[n] = %lld < 0", (long long)nnz);
  FE_ARG(nnz == 0 || colidx != nullptr, "fe_csr_create: colidx is NULL");
  const int64_t ncols = o.ncols > 0 ? o.ncols : n;
  FE_ARG(ncols <= INT32_MAX, "fe_csr_create: ncols = %lld must be below 2^31", (long long)ncols);
  FE_ARG(ncols == n || (o.device_mem_cap_bytes == 0 && !o.transpose && !o.check_symmetric),
         "fe_csr_create: a rectangular matrix (ncols != n) must be resident, without transpose "
         "or symmetry check");
  if (o.validate) FE_TRY(validate_csr(n, ncols, rowptr, colidx));
  if (o.check_symmetric) FE_TRY(check_symmetric(n, rowptr, colidx));
  fe_csr h = new fe_csr_s();
  h->n = n;
  h->ncols = ncols;
  h->nnz = nnz;
  cudaGetDevice(&h->device);
  FE_ARG(o.index_format >= FE_INDEX_AUTO && o.index_format <= FE_INDEX_PACKED,
         "fe_csr_create: index_format = %d", o.index_format);
  const bool packed = o.index_format == FE_INDEX_PACKED;  // resident: plain unless asked
  int tail_max = o.tail_max > 0 ? std::min(o.tail_max, kMaxTailDegree)
                                : (packed ? kDefaultTailMaxPacked : kDefaultTailMax);
  int hub_min = o.hub_min > 0 ? o.hub_min : 4096;
  int hub_chunk = o.hub_chunk > 0 ? o.hub_chunk : 4096;
  if (hub_min < tail_max) hub_min = tail_max;
  int rc;
  FE_ARG(o.l2_persist == 0 || o.l2_persist == 1, "fe_csr_create: l2_persist = %d", o.l2_persist);
  if (o.device_mem_cap_bytes > 0) {
    rc = semiext_create(h, rowptr, colidx, o);
  } else {
    rc = spmm_build_plan(h, rowptr, colidx, tail_max, hub_min, hub_chunk, packed);
    h->plan.l2_persist = o.l2_persist;
  }
  if (rc == FE_OK && o.transpose) {
    std::vector<int64_t> trp;
    std::vector<int32_t> tci;
    transpose_pattern(n, rowptr, colidx, trp, tci);
    fe_csr_opts ot = o;
    ot.transpose = 0;
    ot.validate = 0;
    ot.check_symmetric = 0;
    rc = fe_csr_create_ex(n, trp.data(), tci.data(), &ot, &h->t);
  }
  if (rc != FE_OK) {
    std::string msg = fe_last_error();
    fe_csr_destroy(h);
    set_error(rc, "%s", msg.c_str());
    return rc;
  }
  *out = h;
  return FE_OK;
}

int fe_csr_get_info(fe_csr h, fe_csr_info* info) {
  FE_ARG(h && info, "fe_csr_get_info: NULL argument");
  memset(info, 0, sizeof(*info));
  info->n = h->n;
  info->nnz = h->nnz;
  info->rows_empty = h->rows_empty;
  info->rows_tail = h->rows_tail;
  info->rows_mid = h->rows_mid;
  info->rows_hub = h->rows_hub;
  info->hub_chunks = h->plan.nhub_tasks;
  info->max_degree = h->max_degree;
  info->device_bytes = h->device_bytes + (h->t ? h->t->device_bytes : 0);
  info->semi_external = h->semi_external;
  info->panels = h->semi_external ? semiext_panels(h) : 0;
  info->has_transpose = h->t != nullptr;
  info->tail_max = h->plan.tail_max;
  info->index_format = h->plan.packed ? FE_INDEX_PACKED : FE_INDEX_PLAIN;
  info->index_bytes = h->plan.index_bytes;
  info->ncols = h->ncols;
  return FE_OK;
}

int fe_spmm_t(fe_csr h, const void* X, void* Y, int b, fe_dtype dt) {
  FE_ARG(h != nullptr, "fe_spmm_t: NULL handle");
  FE_ARG(h->t != nullptr, "fe_spmm_t: the handle has no transpose (create it with transpose = 1)");
  return fe_spmm(h->t, X, Y, b, dt);
}

int fe_spmm(fe_csr h, const void* X, void* Y, int b, fe_dtype dt) {
  FE_ARG(h != nullptr, "fe_spmm: NULL handle");
  FE_ARG(X && Y, "fe_spmm: NULL X or Y");
  FE_ARG(is_pow2_le16(b), "fe_spmm: b = %d not in {1,2,4,8,16}", b);
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_spmm: bad dtype %d", (int)dt);
  FE_ARG(((uintptr_t)X % 16) == 0 && ((uintptr_t)Y % 16) == 0, "fe_spmm: X and Y must be 16-byte aligned");
  size_t rowb = (size_t)b * (dt == FE_F32 ? 4 : 8);
  const char* xa = (const char*)X;
  const char* ya = (const char*)Y;
  FE_ARG(xa + rowb * (size_t)h->ncols <= ya || ya + rowb * (size_t)h->n <= xa, "fe_spmm: X and Y overlap");
  if (h->semi_external) return semiext_spmm(h, X, Y, b, dt, cur_stream());
  return spmm_resident(h, X, Y, b, dt, cur_stream());
}

int fe_block_gram_ex(const void* V, int64_t n, int nv, int bv, const void* W, int bw,
                     fe_dtype dt, double alpha, double* G, int engine) {
  FE_ARG(V && W && G, "fe_block_gram: NULL pointer");
  FE_ARG(n >= 1, "fe_block_gram: n < 1");
  FE_ARG(nv >= 1 && nv <= 128, "fe_block_gram: nv = %d not in [1, 128]", nv);
  FE_ARG(is_pow2_le16(bv) && is_pow2_le16(bw), "fe_block_gram: bv, bw must be in {1,2,4,8,16}");
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_block_gram: bad dtype");
  FE_ARG(aligned16(V) && aligned16(W), "fe_block_gram: V and W must be 16-byte aligned");
  BlockSet vs = make_blockset(V, nv, bv, bv, n * bv, dt);
  return gram(vs, n, W, bw, bw, dt, alpha, G, cur_stream(), engine);
}

int fe_block_gram(const void* V, int64_t n, int nv, int bv, const void* W, int bw,
                  fe_dtype dt, double alpha, double* G) {
  return fe_block_gram_ex(V, n, nv, bv, W, bw, dt, alpha, G, FE_ENGINE_AUTO);
}

int fe_block_update(const void* V, int64_t n, int nv, int bv, const double* C, double alpha,
                    double beta, void* W, int bw, fe_dtype dt) {
  return fe_block_update_ex(V, n, nv, bv, C, alpha, beta, W, bw, dt, FE_ENGINE_FMA);
}

int fe_block_update_ex(const void* V, int64_t n, int nv, int bv, const double* C, double alpha,
                       double beta, void* W, int bw, fe_dtype dt, int engine) {
  FE_ARG(W, "fe_block_update: W is NULL");
  FE_ARG(n >= 1, "fe_block_update: n < 1");
  FE_ARG(nv >= 0 && nv <= 128, "fe_block_update: nv = %d not in [0, 128]", nv);
  FE_ARG(nv == 0 || (V && C), "fe_block_update: NULL V or C");
  FE_ARG(is_pow2_le16(bv) && is_pow2_le16(bw), "fe_block_update: bv, bw must be in {1,2,4,8,16}");
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_block_update: bad dtype");
  if (nv > 0) {
    size_t es = dt == FE_F32 ? 4 : 8;
    const char* va = (const char*)V;
    const char* wa = (const char*)W;
    FE_ARG(wa + n * bw * es <= va || va + (size_t)nv * n * bv * es <= wa,
           "fe_block_update: W aliases V");
  }
  FE_ARG(engine == FE_ENGINE_AUTO || engine == FE_ENGINE_FMA || engine == FE_ENGINE_TC,
         "fe_block_update_ex: engine = %d", engine);
  FE_ARG(aligned16(W) && (nv == 0 || aligned16(V)), "fe_block_update: V and W must be 16-byte aligned");
  BlockSet vs = make_blockset(V, nv, bv, bv, n * bv, dt);
  if (engine != FE_ENGINE_FMA) {
    BlockSet ws = make_blockset(W, 1, bw, bw, n * bw, dt);
    const bool tc = dt == FE_F64 && nv >= 1 && tc_combine_supported(vs, ws, dt);
    if (tc) return tc_combine(vs, n, C, bw, ws, cur_stream(), alpha, beta);
    FE_ARG(engine == FE_ENGINE_AUTO,
           "fe_block_update_ex: the tensor-core engine takes FP64 blocks with nv >= 1, bv == bw, "
           "nv*bv <= 64 and bw <= 32");
  }
  return update(vs, n, C, alpha, beta, nullptr, W, bw, bw, dt, cur_stream());
}

int fe_block_combine(const void* V, int64_t n, int nv, int bv, const double* Y, int nout, void* Out,
                     fe_dtype dt, int engine) {
  FE_ARG(V && Y && Out, "fe_block_combine: NULL pointer");
  FE_ARG(n >= 1, "fe_block_combine: n < 1");
  FE_ARG(nv >= 1 && nv <= 128, "fe_block_combine: nv = %d not in [1, 128]", nv);
  FE_ARG(nout >= 1 && nout <= 128, "fe_block_combine: nout = %d not in [1, 128]", nout);
  FE_ARG(is_pow2_le16(bv), "fe_block_combine: bv = %d not in {1,2,4,8,16}", bv);
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_block_combine: bad dtype");
  {
    const size_t es = dt == FE_F32 ? 4 : 8;
    const char* va = (const char*)V;
    const char* oa = (const char*)Out;
    FE_ARG(oa + (size_t)nout * n * bv * es <= va || va + (size_t)nv * n * bv * es <= oa,
           "fe_block_combine: Out aliases V");
  }
  FE_ARG(aligned16(V) && aligned16(Out), "fe_block_combine: V and Out must be 16-byte aligned");
  BlockSet vs = make_blockset(V, nv, bv, bv, n * bv, dt);
  BlockSet os = make_blockset(Out, nout, bv, bv, n * bv, dt);
  return combine(vs, n, Y, nout * bv, os, dt, cur_stream(), engine);
}

int fe_block_update_gram(const void* V, int64_t n, int nv, int b, const double* C, double alpha,
                         double beta, void* W, fe_dtype dt, double* G) {
  FE_ARG(W && G, "fe_block_update_gram: NULL W or G");
  FE_ARG(n >= 1, "fe_block_update_gram: n < 1");
  FE_ARG(nv >= 0 && nv <= 128, "fe_block_update_gram: nv = %d not in [0, 128]", nv);
  FE_ARG(nv == 0 || (V && C), "fe_block_update_gram: NULL V or C");
  FE_ARG(b == 1 || b == 2 || b == 4 || b == 8, "fe_block_update_gram: b = %d not in {1,2,4,8}", b);
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_block_update_gram: bad dtype");
  if (nv > 0) {
    size_t es = dt == FE_F32 ? 4 : 8;
    const char* va = (const char*)V;
    const char* wa = (const char*)W;
    FE_ARG(wa + n * b * es <= va || va + (size_t)nv * n * b * es <= wa,
           "fe_block_update_gram: W aliases V");
  }
  FE_ARG(aligned16(W) && (nv == 0 || aligned16(V)), "fe_block_update_gram: V and W must be 16-byte aligned");
  BlockSet vs = make_blockset(V, nv, b, b, n * b, dt);
  return update_gram(vs, n, C, alpha, beta, nullptr, W, b, dt, 1, nullptr, G, cur_stream());
}

int fe_block_orth(const void* V, int64_t n, int nv, int b, void* W, fe_dtype dt, double anorm,
                  uint64_t seed, double* G, double* R, int* replaced) {
  FE_ARG(W && R, "fe_block_orth: NULL W or R");
  FE_ARG(nv == 0 || (V && G), "fe_block_orth: NULL V or G");
  FE_ARG(n >= 1 && nv >= 0 && nv <= 128, "fe_block_orth: bad n or nv");
  FE_ARG(is_pow2_le16(b), "fe_block_orth: b must be in {1,2,4,8,16}");
  FE_ARG((int64_t)(nv + 1) * b <= n, "fe_block_orth: (nv+1)*b > n");
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_block_orth: bad dtype");
  FE_ARG(aligned16(W) && (nv == 0 || aligned16(V)), "fe_block_orth: V and W must be 16-byte aligned");
  BlockSet vs = make_blockset(V, nv, b, b, n * b, dt);
  DevBuf an;
  FE_TRY(an.alloc(sizeof(double)));
  cudaStream_t s = cur_stream();
  double a = anorm > 0 ? anorm : 0.0;
  FE_CUDA(cudaMemcpyAsync(an.p, &a, sizeof(double), cudaMemcpyHostToDevice, s));
  uint64_t counter = 0;
  int rep = 0;
  DevBuf gdummy;
  if (nv == 0) {
    FE_TRY(gdummy.alloc(sizeof(double) * b));
    G = gdummy.as<double>();
  }
  int rc = orth(vs, n, W, b, dt, an.as<double>(), a, seed, &counter, G, b, R, b, &rep, s);
  if (replaced) *replaced = rep;
  if (rc == FE_OK) FE_CUDA(cudaStreamSynchronize(s));
  return rc;
}

int fe_random_normal(void* X, int64_t n, int b, fe_dtype dt, uint64_t seed, uint64_t stream,
                     uint64_t offset) {
  FE_ARG(X, "fe_random_normal: X is NULL");
  FE_ARG(n >= 1 && b >= 1 && b <= 64, "fe_random_normal: bad n or b");
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_random_normal: bad dtype");
  return random_normal(X, n, b, b, dt, seed, stream, offset, cur_stream());
}

}  // extern "C"
