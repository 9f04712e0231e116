// Semi-external SpMM (Section 3.3: the sparse matrix streams in from SSDs while the dense
// blocks stay in memory; here pinned host memory plays the SSDs and HBM plays RAM).
//
// At create time the rows are cut into panels whose packed plan (column indices, tail slices,
// warp tasks, hub lists -- the same layout the resident SpMM uses, with panel-local column
// offsets) fits half of the device-memory cap.  Each fe_spmm streams the panels through two
// device buffers: panel p+1 is copied on a copy stream while the kernels of panel p run
// (double buffering; the paper's asynchronous I/O of the next partition while the current
// one is multiplied, Section 3.3.3).  Events order buffer reuse.  The host then waits for
// the last panel for at most copy_timeout_ms and returns FE_ERR_TIMEOUT past that bound.
// The streamed bytes bound this mode (pinned copies run at ~210 GB/s on a GB300 node), so by
// default the warp-task rows' column indices travel bit-packed as gaps (index_format), about
// 0.55-0.65 of the int32 bytes on R-MAT graphs.  A handle's transpose (fe_svds) streams its
// own panels the same way.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

struct PanelInfo {
  int64_t r0, r1, nnz;
  int64_t index_words;  // plain: task column indices; packed: gap bit-stream words
  size_t off_colidx, off_slice_rows, off_ell, off_tasks, off_hub_rows, off_hub_begin, bytes;
  size_t host_off;  // offset of the packed panel in the pinned arena
  int nbuckets;
  int32_t deg_of_bucket[kMaxBuckets], deg_slice_begin[kMaxBuckets];
  int64_t deg_ell_base[kMaxBuckets];
  int64_t nslices, ntasks, nhub_tasks, nhub;
};

struct SemiExt {
  std::vector<PanelInfo> panels;
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
  void* dbuf[2] = {nullptr, nullptr};
  size_t dbuf_bytes = 0;
  DevBuf partials;
  cudaStream_t copy = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr}, done = nullptr;
  int timeout_ms = 60000;
  bool packed = false;   // task rows' columns as bit-packed gaps (index_format)
  bool direct = false;   // kernels read the pinned panels through their device mapping
  bool pending = false;  // a previous call returned FE_ERR_TIMEOUT with work in flight
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes row i adds to a panel (estimate used to cut panels): its column indices in the plan's
// format, plus its slice row id or its task records.
static size_t row_bytes(const int32_t* cols, int64_t d, int tail_max, int hub_min, int hub_chunk,
                        bool packed) {
  size_t b = plan_row_index_bytes(cols, d, tail_max, hub_chunk, packed);
  if (d <= tail_max) b += 4;
  else if (d <= hub_min) b += sizeof(Task);
  else b += sizeof(Task) * (size_t)ceil_div(d, hub_chunk) + 8;
  return b;
}

static int wait_event(cudaEvent_t e, int timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) return FE_OK;
    if (q != cudaErrorNotReady) return cuda_fail(q, "cudaEventQuery", __FILE__, __LINE__);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms > timeout_ms)
      return set_error(FE_ERR_TIMEOUT, "semi-external SpMM: panels not done after %d ms", timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// Worst-case padding of one panel's slices: every degree bucket's last 32-row slice may hold a
// single row, so 31 padded lanes of ELL indices plus 31 row ids per bucket.
static size_t slice_padding(int tail_max) {
  return (size_t)4 * 31 * ((size_t)tail_max * (tail_max + 1) / 2 + (size_t)tail_max + 1);
}

int semiext_create(fe_csr h, const int64_t* rowptr, const int32_t* colidx, const fe_csr_opts& o) {
  const int64_t n = h->n;
  // index format: packed gaps unless the caller asks for plain indices (the streamed bytes are
  // what bound this mode)
  const bool packed = o.index_format != FE_INDEX_PLAIN;
  int tail_max = o.tail_max > 0 ? std::min(o.tail_max, kMaxTailDegree)
                                : (packed ? kDefaultTailMaxPacked : kDefaultTailMax);
  if (o.tail_max <= 0) {
    // default cutoff: keep the slice padding below 1/8 of a panel buffer
    const size_t half = o.device_mem_cap_bytes > 0 ? (size_t)o.device_mem_cap_bytes / 2 : 0;
    while (tail_max > 4 && slice_padding(tail_max) * 8 > half) tail_max /= 2;
  }
  int hub_min = o.hub_min > 0 ? o.hub_min : 4096;
  const int hub_chunk = o.hub_chunk > 0 ? o.hub_chunk : 4096;
  if (hub_min < tail_max) hub_min = tail_max;
  const int64_t cap = o.device_mem_cap_bytes;
  // resident size: the plan (task column indices, ELL slices, tasks); if it fits, stay resident
  // resident size with plain indices (an upper bound for a packed resident plan)
  size_t resident = 64 * 1024;
  int64_t max_hub_tasks = 0;
  #pragma omp parallel for schedule(static) reduction(+ : resident, max_hub_tasks)
  for (int64_t i = 0; i < n; ++i) {
    const int64_t d = rowptr[i + 1] - rowptr[i];
    resident += row_bytes(colidx + rowptr[i], d, tail_max, hub_min, hub_chunk, false) + 4;
    if (d > hub_min) max_hub_tasks += ceil_div(d, hub_chunk);
  }
  resident += 16 * 8 * (size_t)max_hub_tasks;
  if ((int64_t)resident <= cap)
    return spmm_build_plan(h, rowptr, colidx, tail_max, hub_min, hub_chunk,
                           o.index_format == FE_INDEX_PACKED);
  std::vector<uint32_t> rbytes(n);
  #pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < n; ++i) {
    const int64_t d = rowptr[i + 1] - rowptr[i];
    rbytes[i] = (uint32_t)std::min<size_t>(
        row_bytes(colidx + rowptr[i], d, tail_max, hub_min, hub_chunk, packed) + 4 + 64, UINT32_MAX);
  }

  SemiExt* sx = new SemiExt();
  h->sx = sx;
  h->plan.tail_max = tail_max;
  h->semi_external = 1;
  sx->timeout_ms = o.copy_timeout_ms > 0 ? o.copy_timeout_ms : 60000;
  sx->direct = o.semi_direct != 0;
  sx->packed = packed;
  h->plan.packed = packed ? 1 : 0;
  // cut panels: packed size <= target and nnz <= panel_nnz
  // hub partials + slack
  const size_t reserve = 16 * 8 * (size_t)std::min<int64_t>(max_hub_tasks, 1 << 20) + (64 << 10);
  FE_ARG(cap > (int64_t)reserve + (1 << 16), "device_mem_cap_bytes = %lld is too small", (long long)cap);
  const size_t pad = slice_padding(tail_max);
  FE_ARG((size_t)cap > reserve + 2 * pad + (1 << 16),
         "device_mem_cap_bytes = %lld is too small for tail_max = %d", (long long)cap, tail_max);
  const size_t target = ((size_t)cap - reserve) / 2 - pad;
  const int64_t panel_nnz = o.panel_nnz > 0 ? o.panel_nnz : ((int64_t)64 << 20);
  std::vector<std::pair<int64_t, int64_t>> ranges;
  {
    int64_t r0 = 0;
    size_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
      const size_t rb = rbytes[i];
      if (i > r0 && (acc + rb > target || rowptr[i + 1] - rowptr[r0] > panel_nnz)) {
        ranges.push_back({r0, i});
        r0 = i;
        acc = 0;
      }
      acc += rb;
    }
    ranges.push_back({r0, n});
  }
  // build each panel's plan and pack it
  std::vector<HostPlan> plans(ranges.size());
  size_t total = 0, maxbytes = 0;
  int64_t maxhub = 0;
  for (size_t p = 0; p < ranges.size(); ++p) {
    HostPlan& hp = plans[p];
    FE_TRY(build_host_plan(rowptr, colidx, ranges[p].first, ranges[p].second, tail_max, hub_min,
                           hub_chunk, packed, hp));
    PanelInfo pi;
    memset(&pi, 0, sizeof(pi));
    pi.r0 = ranges[p].first;
    pi.r1 = ranges[p].second;
    pi.nnz = rowptr[pi.r1] - rowptr[pi.r0];
    size_t off = 0;
    pi.index_words = packed ? (int64_t)hp.tbits.size() : hp.tcol_total;
    pi.off_colidx = off; off = align256(off + 4 * (size_t)pi.index_words);
    h->plan.index_bytes += 4 * (pi.index_words + hp.ell_total);
    pi.off_slice_rows = off; off = align256(off + 4 * hp.slice_rows.size());
    pi.off_ell = off; off = align256(off + 4 * (size_t)hp.ell_total);
    pi.off_tasks = off; off = align256(off + (packed ? sizeof(PTask) : sizeof(Task)) * (size_t)hp.ntasks);
    pi.off_hub_rows = off; off = align256(off + 4 * (size_t)hp.nhub);
    pi.off_hub_begin = off; off = align256(off + 4 * (size_t)(hp.nhub + 1));
    pi.bytes = off;
    pi.host_off = total;
    total += off;
    maxbytes = std::max(maxbytes, off);
    maxhub = std::max(maxhub, hp.nhub_tasks);
    pi.nbuckets = hp.nbuckets;
    for (int i = 0; i < hp.nbuckets; ++i) {
      pi.deg_of_bucket[i] = hp.deg_of_bucket[i];
      pi.deg_slice_begin[i] = hp.deg_slice_begin[i];
      pi.deg_ell_base[i] = hp.deg_ell_base[i];
    }
    pi.nslices = hp.nslices;
    pi.ntasks = hp.ntasks;
    pi.nhub_tasks = hp.nhub_tasks;
    pi.nhub = hp.nhub;
    h->max_degree = std::max(h->max_degree, hp.max_degree);
    h->rows_empty += hp.rows_empty;
    h->rows_tail += hp.rows_tail;
    h->rows_mid += hp.rows_mid;
    h->rows_hub += hp.rows_hub;
    sx->panels.push_back(pi);
  }
  const size_t need = 2 * maxbytes + 16 * 8 * (size_t)std::max<int64_t>(maxhub, 1);
  FE_ARG((int64_t)need <= cap,
         "device_mem_cap_bytes = %lld cannot hold two panel buffers (%zu bytes needed)", (long long)cap, need);
  cudaError_t e = cudaMallocHost((void**)&sx->pinned, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sx->pinned = nullptr;
    return set_error(FE_ERR_OOM, "cudaMallocHost(%zu) for the semi-external CSR failed", total);
  }
  sx->pinned_bytes = total;
  for (size_t p = 0; p < plans.size(); ++p) {
    const PanelInfo& pi = sx->panels[p];
    const HostPlan& hp = plans[p];
    char* base = sx->pinned + pi.host_off;
    if (packed) memcpy(base + pi.off_colidx, hp.tbits.data(), 4 * (size_t)pi.index_words);
    else memcpy(base + pi.off_colidx, hp.tcol.data(), 4 * (size_t)pi.index_words);
    memcpy(base + pi.off_slice_rows, hp.slice_rows.data(), 4 * hp.slice_rows.size());
    memcpy(base + pi.off_ell, hp.ell.data(), 4 * (size_t)hp.ell_total);
    if (packed) memcpy(base + pi.off_tasks, hp.ptasks.data(), sizeof(PTask) * (size_t)hp.ntasks);
    else memcpy(base + pi.off_tasks, hp.tasks.data(), sizeof(Task) * (size_t)hp.ntasks);
    memcpy(base + pi.off_hub_rows, hp.hub_rows.data(), 4 * (size_t)hp.nhub);
    memcpy(base + pi.off_hub_begin, hp.hub_task_begin.data(), 4 * (size_t)(hp.nhub + 1));
  }
  plans.clear();
  sx->dbuf_bytes = maxbytes;
  for (int k = 0; k < 2 && !sx->direct; ++k) {
    e = cudaMalloc(&sx->dbuf[k], maxbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      sx->dbuf[k] = nullptr;
      return set_error(FE_ERR_OOM, "cudaMalloc(%zu) for a panel buffer failed", maxbytes);
    }
  }
  FE_TRY(sx->partials.alloc(16 * 8 * (size_t)std::max<int64_t>(maxhub, 1)));
  h->device_bytes = (sx->direct ? 0 : 2 * (int64_t)maxbytes) + (int64_t)sx->partials.bytes;
  FE_CUDA(cudaStreamCreateWithFlags(&sx->copy, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    FE_CUDA(cudaEventCreateWithFlags(&sx->copied[k], cudaEventDisableTiming));
    FE_CUDA(cudaEventCreateWithFlags(&sx->consumed[k], cudaEventDisableTiming));
  }
  FE_CUDA(cudaEventCreateWithFlags(&sx->done, cudaEventDisableTiming));
  return FE_OK;
}

int semiext_spmm(fe_csr h, const void* X, void* Y, int b, fe_dtype dt, cudaStream_t s) {
  SemiExt* sx = h->sx;
  if (sx->pending) {
    FE_TRY(wait_event(sx->done, sx->timeout_ms));
    sx->pending = false;
  }
  for (size_t p = 0; p < sx->panels.size(); ++p) {
    const PanelInfo& pi = sx->panels[p];
    const int k = (int)(p & 1);
    const char* base;
    if (sx->direct) {
      // pinned memory is mapped into the device address space (unified addressing)
      base = sx->pinned + pi.host_off;
    } else {
      // the buffer is free once the kernels of panel p-2 are done
      FE_CUDA(cudaStreamWaitEvent(sx->copy, sx->consumed[k], 0));
      FE_CUDA(cudaMemcpyAsync(sx->dbuf[k], sx->pinned + pi.host_off, pi.bytes, cudaMemcpyHostToDevice, sx->copy));
      FE_CUDA(cudaEventRecord(sx->copied[k], sx->copy));
      FE_CUDA(cudaStreamWaitEvent(s, sx->copied[k], 0));
      base = static_cast<const char*>(sx->dbuf[k]);
    }
    PlanView v;
    memset(&v, 0, sizeof(v));
    v.colidx = reinterpret_cast<const int32_t*>(base + pi.off_colidx);
    v.tbits = reinterpret_cast<const uint32_t*>(base + pi.off_colidx);
    v.packed = sx->packed ? 1 : 0;
    v.tasks = base + pi.off_tasks;
    v.ntasks = pi.ntasks;
    v.nhub_tasks = pi.nhub_tasks;
    v.slice_rows = reinterpret_cast<const int32_t*>(base + pi.off_slice_rows);
    v.ell = reinterpret_cast<const int32_t*>(base + pi.off_ell);
    v.nslices = pi.nslices;
    v.nbuckets = pi.nbuckets;
    for (int i = 0; i < pi.nbuckets; ++i) {
      v.deg_of_bucket[i] = pi.deg_of_bucket[i];
      v.deg_slice_begin[i] = pi.deg_slice_begin[i];
      v.deg_ell_base[i] = pi.deg_ell_base[i];
    }
    v.hub_rows = reinterpret_cast<const int32_t*>(base + pi.off_hub_rows);
    v.hub_task_begin = reinterpret_cast<const int32_t*>(base + pi.off_hub_begin);
    v.nhub = pi.nhub;
    FE_TRY(spmm_view(v, X, Y, sx->partials.p, b, dt, s));
    FE_CUDA(cudaEventRecord(sx->consumed[k], s));
  }
  FE_CUDA(cudaEventRecord(sx->done, s));
  const int rc = wait_event(sx->done, sx->timeout_ms);
  if (rc == FE_ERR_TIMEOUT) sx->pending = true;
  return rc;
}

void semiext_destroy(fe_csr h) {
  SemiExt* sx = h->sx;
  if (!sx) return;
  if (sx->copy) cudaStreamSynchronize(sx->copy);
  cudaDeviceSynchronize();
  for (int k = 0; k < 2; ++k) {
    if (sx->dbuf[k]) cudaFree(sx->dbuf[k]);
    if (sx->copied[k]) cudaEventDestroy(sx->copied[k]);
    if (sx->consumed[k]) cudaEventDestroy(sx->consumed[k]);
  }
  if (sx->done) cudaEventDestroy(sx->done);
  if (sx->copy) cudaStreamDestroy(sx->copy);
  if (sx->pinned) cudaFreeHost(sx->pinned);
  delete sx;
  h->sx = nullptr;
}

int64_t semiext_panels(fe_csr h) { return h->sx ? (int64_t)h->sx->panels.size() : 0; }

}  // namespace fe
