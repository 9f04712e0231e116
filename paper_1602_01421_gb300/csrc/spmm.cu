// SpMM, Y = A X for a 0/1 pattern matrix A (Section 3.3): every non-zero (i, j) adds row j
// of the dense block X to row i of Y.  X and Y are row-major n x b (Section 3.3.2).
//
// GB300 layout of A, built once per handle from the CSR (Section 3.3.1 / 3.3.3 motives: the
// paper fights branchy single-entry rows with SCSR+COO tiles and power-law load imbalance
// with work stealing; here the same two problems are solved by degree binning):
//   * tail rows (degree <= tail_max, 85% of R-MAT rows): grouped by degree into 32-row
//     slices whose column indices are stored transposed ("SELL-32"): lane l of a warp owns
//     row l of the slice and step t loads ell[t*32 + l], one coalesced 128-byte load per
//     step and no divergence, since all 32 rows of a slice have the same degree;
//   * mid rows (tail_max < degree <= hub_min): one warp per row (a "task"), 32 consecutive
//     column indices per coalesced load, each lane gathering 16 bytes of an X row;
//   * hub rows (degree > hub_min): split into tasks of hub_chunk non-zeros; each task writes
//     a partial row, and a second kernel adds a hub's partials in task order (deterministic,
//     no atomics).
// Tasks are ordered longest first so the block scheduler handles them like a longest-
// processing-time list; tail slices follow in the same launch.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fe_internal.cuh"
#include "vec.cuh"

namespace fe {

struct Task {
  int64_t start;  // offset into colidx
  int32_t row;    // output row
  int32_t len;    // non-zeros
};
static_assert(sizeof(Task) == 16, "Task must be 16 bytes");

// Per (type, b) geometry: a lane moves NE elements (<= 16 bytes) per load; an X row of
// b elements spans C lanes in a warp task (P = 32 / C rows gathered per warp instruction)
// and NCH = C chunks in a tail lane.
template <typename T, int B>
struct Geo {
  static constexpr int ROWB = B * (int)sizeof(T);
  static constexpr int NE = ROWB <= 16 ? B : 16 / (int)sizeof(T);
  static constexpr int C = B / NE;
  static constexpr int P = 32 / C;
  static constexpr int UNROLL = C >= 4 ? 1 : 4 / C;
};

constexpr int kMaxBuckets = 34;
struct SpmmParams {
  const int32_t* colidx;
  const Task* tasks;
  int64_t ntasks, nhub_tasks, task_ctas;
  const int32_t* slice_rows;
  const int32_t* ell;
  int64_t nslices;
  int nbuckets;
  int32_t bucket_deg[kMaxBuckets];
  int32_t bucket_slice_begin[kMaxBuckets + 1];
  int64_t bucket_ell_base[kMaxBuckets];
};

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 8;

template <typename T, int B>
__device__ __forceinline__ void run_task(const SpmmParams& p, int64_t ti, const T* __restrict__ X,
                                         T* __restrict__ Y, T* __restrict__ partial, int lane) {
  using G = Geo<T, B>;
  const int4 raw = __ldg(reinterpret_cast<const int4*>(p.tasks + ti));
  const int64_t start = (int64_t)(uint32_t)raw.x | ((int64_t)raw.y << 32);
  const int row = raw.z;
  const int len = raw.w;
  const int chunk = lane % G::C;
  const int slot = lane / G::C;
  T acc[G::NE];
#pragma unroll
  for (int e = 0; e < G::NE; ++e) acc[e] = T(0);
  const int32_t* __restrict__ ci = p.colidx + start;
  for (int base = 0; base < len; base += 32 * G::UNROLL) {
    int cols[G::UNROLL];
#pragma unroll
    for (int u = 0; u < G::UNROLL; ++u) {
      int k = base + u * 32 + lane;
      cols[u] = k < len ? __ldcs(ci + k) : -1;
    }
#pragma unroll
    for (int u = 0; u < G::UNROLL; ++u) {
#pragma unroll
      for (int g = 0; g < 32; g += G::P) {
        int col = __shfl_sync(kFull, cols[u], g + slot);
        if (col >= 0) {
          T f[G::NE];
          ld_frag<T, G::NE>(X + (int64_t)col * B + chunk * G::NE, f);
#pragma unroll
          for (int e = 0; e < G::NE; ++e) acc[e] += f[e];
        }
      }
    }
  }
  // tree-reduce the P slot partials of each chunk (lanes that differ above the chunk bits)
#pragma unroll
  for (int off = G::C; off < 32; off <<= 1)
#pragma unroll
    for (int e = 0; e < G::NE; ++e) acc[e] += __shfl_xor_sync(kFull, acc[e], off);
  if (slot == 0) {
    T* dst = ti < p.nhub_tasks ? partial + ti * B : Y + (int64_t)row * B;
    st_frag<T, G::NE>(dst + chunk * G::NE, acc);
  }
}

template <typename T, int B>
__device__ __forceinline__ void run_slice(const SpmmParams& p, int64_t si, const T* __restrict__ X,
                                          T* __restrict__ Y, int lane) {
  using G = Geo<T, B>;
  int bkt = 0;
  while (bkt + 1 < p.nbuckets && si >= p.bucket_slice_begin[bkt + 1]) ++bkt;
  const int deg = p.bucket_deg[bkt];
  const int64_t off = p.bucket_ell_base[bkt] + (si - p.bucket_slice_begin[bkt]) * 32 * (int64_t)deg;
  const int row = __ldcs(p.slice_rows + si * 32 + lane);
  T acc[B];
#pragma unroll
  for (int e = 0; e < B; ++e) acc[e] = T(0);
  const int32_t* __restrict__ e = p.ell + off + lane;
  int t = 0;
  for (; t + 4 <= deg; t += 4) {
    int c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = __ldcs(e + (t + u) * 32);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int ch = 0; ch < G::C; ++ch) {
        T f[G::NE];
        ld_frag<T, G::NE>(X + (int64_t)c[u] * B + ch * G::NE, f);
#pragma unroll
        for (int q = 0; q < G::NE; ++q) acc[ch * G::NE + q] += f[q];
      }
  }
  for (; t < deg; ++t) {
    int c = __ldcs(e + t * 32);
#pragma unroll
    for (int ch = 0; ch < G::C; ++ch) {
      T f[G::NE];
      ld_frag<T, G::NE>(X + (int64_t)c * B + ch * G::NE, f);
#pragma unroll
      for (int q = 0; q < G::NE; ++q) acc[ch * G::NE + q] += f[q];
    }
  }
  if (row >= 0) {
#pragma unroll
    for (int ch = 0; ch < G::C; ++ch) st_frag<T, G::NE>(Y + (int64_t)row * B + ch * G::NE, acc + ch * G::NE);
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(256) spmm_main_kernel(const SpmmParams p, const T* __restrict__ X,
                                                        T* __restrict__ Y, T* __restrict__ partial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((int64_t)blockIdx.x < p.task_ctas) {
    const int64_t ti = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    if (ti < p.ntasks) run_task<T, B>(p, ti, X, Y, partial, lane);
  } else {
    const int64_t si = ((int64_t)blockIdx.x - p.task_ctas) * kWarpsPerCta + warp;
    if (si < p.nslices) run_slice<T, B>(p, si, X, Y, lane);
  }
}

// Y[hub_rows[h]] = sum of the hub's task partials in task order.
template <typename T, int B>
__global__ void hub_reduce_kernel(const int32_t* __restrict__ hub_rows,
                                  const int32_t* __restrict__ hub_task_begin, int64_t nhub,
                                  const T* __restrict__ partial, T* __restrict__ Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nhub * B) return;
  const int64_t h = i / B;
  const int c = (int)(i % B);
  T s = T(0);
  for (int t = hub_task_begin[h]; t < hub_task_begin[h + 1]; ++t) s += partial[(int64_t)t * B + c];
  Y[(int64_t)hub_rows[h] * B + c] = s;
}

template <typename T, int B>
static int launch_spmm(fe_csr h, const T* X, T* Y, cudaStream_t s) {
  const fe_spmm_plan& pl = h->plan;
  SpmmParams p;
  memset(&p, 0, sizeof(p));
  p.colidx = h->d_colidx;
  p.tasks = reinterpret_cast<const Task*>(pl.d_tasks);
  p.ntasks = pl.ntasks;
  p.nhub_tasks = pl.nhub_tasks;
  p.task_ctas = ceil_div(pl.ntasks, kWarpsPerCta);
  p.slice_rows = pl.d_slice_rows;
  p.ell = pl.d_ell;
  p.nslices = pl.nslices;
  p.nbuckets = pl.nbuckets;
  for (int i = 0; i < pl.nbuckets; ++i) {
    p.bucket_deg[i] = pl.deg_of_bucket[i];
    p.bucket_slice_begin[i] = pl.deg_slice_begin[i];
    p.bucket_ell_base[i] = pl.deg_ell_base[i];
  }
  p.bucket_slice_begin[pl.nbuckets] = (int32_t)pl.nslices;
  const int64_t ctas = p.task_ctas + ceil_div(pl.nslices, kWarpsPerCta);
  if (ctas > 0) {
    spmm_main_kernel<T, B><<<(unsigned)ctas, 256, 0, s>>>(p, X, Y, h->partials.as<T>());
    count_launch();
    FE_CUDA(cudaGetLastError());
  }
  if (pl.nhub > 0) {
    const int64_t th = pl.nhub * B;
    hub_reduce_kernel<T, B><<<(unsigned)ceil_div(th, 256), 256, 0, s>>>(
        pl.d_hub_rows, pl.d_hub_task_begin, pl.nhub, h->partials.as<T>(), Y);
    count_launch();
    FE_CUDA(cudaGetLastError());
  }
  return FE_OK;
}

int spmm_resident(fe_csr h, const void* X, void* Y, int b, fe_dtype dt, cudaStream_t s) {
  if (dt == FE_F32) {
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    switch (b) {
      case 1: return launch_spmm<float, 1>(h, x, y, s);
      case 2: return launch_spmm<float, 2>(h, x, y, s);
      case 4: return launch_spmm<float, 4>(h, x, y, s);
      case 8: return launch_spmm<float, 8>(h, x, y, s);
      case 16: return launch_spmm<float, 16>(h, x, y, s);
    }
  } else {
    const double* x = static_cast<const double*>(X);
    double* y = static_cast<double*>(Y);
    switch (b) {
      case 1: return launch_spmm<double, 1>(h, x, y, s);
      case 2: return launch_spmm<double, 2>(h, x, y, s);
      case 4: return launch_spmm<double, 4>(h, x, y, s);
      case 8: return launch_spmm<double, 8>(h, x, y, s);
      case 16: return launch_spmm<double, 16>(h, x, y, s);
    }
  }
  return set_error(FE_ERR_INVALID, "spmm: unsupported b = %d", b);
}

// ---------------------------------------------------------------- plan (host, at create)

static int dev_upload(fe_csr h, void** dst, const void* src, size_t bytes) {
  *dst = nullptr;
  if (bytes == 0) return FE_OK;
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return set_error(FE_ERR_OOM, "cudaMalloc(%zu) for the CSR failed: %s", bytes, cudaGetErrorString(e));
  }
  h->allocations.push_back(*dst);
  h->device_bytes += (int64_t)bytes;
  if (src) FE_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return FE_OK;
}

int spmm_build_plan(fe_csr h, const int64_t* rowptr, const int32_t* colidx, int tail_max,
                    int hub_min, int hub_chunk) {
  const int64_t n = h->n;
  fe_spmm_plan& pl = h->plan;
  pl.tail_max = tail_max;
  pl.hub_min = hub_min;
  pl.hub_chunk = hub_chunk;
  int64_t maxdeg = 0;
  std::vector<int64_t> tail_cnt(tail_max + 1, 0);
  std::vector<int64_t> mid_cnt(hub_min + 1, 0);
  int64_t nhub = 0, nhub_tasks = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = rowptr[i + 1] - rowptr[i];
    maxdeg = std::max(maxdeg, d);
    if (d <= tail_max) tail_cnt[d]++;
    else if (d <= hub_min) mid_cnt[d]++;
    else { nhub++; nhub_tasks += ceil_div(d, hub_chunk); }
  }
  h->max_degree = maxdeg;
  h->rows_empty = tail_cnt[0];
  h->rows_tail = 0;
  for (int d = 1; d <= tail_max; ++d) h->rows_tail += tail_cnt[d];
  h->rows_mid = 0;
  for (int d = tail_max + 1; d <= hub_min; ++d) h->rows_mid += mid_cnt[d];
  h->rows_hub = nhub;
  FE_ARG(nhub_tasks < INT32_MAX, "spmm plan: too many hub tasks");

  // ---- tail slices: buckets by degree, descending, empty bucket dropped
  pl.nbuckets = 0;
  int64_t nslices = 0, ell_total = 0;
  std::vector<int> bucket_of_deg(tail_max + 1, -1);
  for (int d = tail_max; d >= 0; --d) {
    if (tail_cnt[d] == 0) continue;
    int bk = pl.nbuckets++;
    bucket_of_deg[d] = bk;
    pl.deg_of_bucket[bk] = d;
    pl.deg_slice_begin[bk] = (int32_t)nslices;
    pl.deg_ell_base[bk] = ell_total;
    int64_t sl = ceil_div(tail_cnt[d], 32);
    nslices += sl;
    ell_total += sl * 32 * d;
  }
  FE_ARG(nslices < INT32_MAX, "spmm plan: too many tail slices");
  pl.nslices = nslices;
  std::vector<int32_t> slice_rows(nslices * 32, -1);
  std::vector<int64_t> cursor(tail_max + 1, 0);
  for (int d = 0; d <= tail_max; ++d)
    if (bucket_of_deg[d] >= 0) cursor[d] = (int64_t)pl.deg_slice_begin[bucket_of_deg[d]] * 32;
  // ---- tasks: hub chunks first, then mid rows by degree descending (stable in row order)
  std::vector<int64_t> mid_pos(hub_min + 2, 0);
  {
    int64_t acc = nhub_tasks;
    for (int d = hub_min; d > tail_max; --d) { mid_pos[d] = acc; acc += mid_cnt[d]; }
  }
  const int64_t ntasks = nhub_tasks + h->rows_mid;
  std::vector<Task> tasks(ntasks);
  std::vector<int32_t> hub_rows(nhub), hub_begin(nhub + 1);
  int64_t ht = 0, hi = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = rowptr[i + 1] - rowptr[i];
    if (d <= tail_max) {
      slice_rows[cursor[d]++] = (int32_t)i;
    } else if (d <= hub_min) {
      tasks[mid_pos[d]++] = Task{rowptr[i], (int32_t)i, (int32_t)d};
    } else {
      hub_rows[hi] = (int32_t)i;
      hub_begin[hi] = (int32_t)ht;
      for (int64_t c = 0; c < d; c += hub_chunk)
        tasks[ht++] = Task{rowptr[i] + c, (int32_t)i, (int32_t)std::min<int64_t>(hub_chunk, d - c)};
      ++hi;
    }
  }
  hub_begin[nhub] = (int32_t)ht;
  pl.ntasks = ntasks;
  pl.nhub_tasks = nhub_tasks;
  pl.nhub = nhub;
  // ---- ELL fill (transposed per slice; padding lanes read column 0 and are not written)
  std::vector<int32_t> ell(ell_total > 0 ? ell_total : 1, 0);
  for (int bk = 0; bk < pl.nbuckets; ++bk) {
    const int d = pl.deg_of_bucket[bk];
    if (d == 0) continue;
    const int64_t s0 = pl.deg_slice_begin[bk];
    const int64_t s1 = (bk + 1 < pl.nbuckets) ? pl.deg_slice_begin[bk + 1] : nslices;
    #pragma omp parallel for schedule(static)
    for (int64_t s = s0; s < s1; ++s) {
      int32_t* e = ell.data() + pl.deg_ell_base[bk] + (s - s0) * 32 * d;
      for (int lane = 0; lane < 32; ++lane) {
        int32_t r = slice_rows[s * 32 + lane];
        for (int t = 0; t < d; ++t) e[t * 32 + lane] = r >= 0 ? colidx[rowptr[r] + t] : 0;
      }
    }
  }
  // ---- upload
  FE_TRY(dev_upload(h, (void**)&h->d_rowptr, rowptr, sizeof(int64_t) * (n + 1)));
  FE_TRY(dev_upload(h, (void**)&h->d_colidx, colidx, sizeof(int32_t) * h->nnz));
  FE_TRY(dev_upload(h, (void**)&pl.d_slice_rows, slice_rows.data(), sizeof(int32_t) * slice_rows.size()));
  FE_TRY(dev_upload(h, (void**)&pl.d_ell, ell.data(), sizeof(int32_t) * ell_total));
  FE_TRY(dev_upload(h, &pl.d_tasks, tasks.data(), sizeof(Task) * ntasks));
  FE_TRY(dev_upload(h, (void**)&pl.d_hub_rows, hub_rows.data(), sizeof(int32_t) * nhub));
  FE_TRY(dev_upload(h, (void**)&pl.d_hub_task_begin, hub_begin.data(), sizeof(int32_t) * (nhub + 1)));
  if (nhub_tasks > 0) {
    FE_TRY(h->partials.alloc(sizeof(double) * 16 * nhub_tasks));
    h->device_bytes += (int64_t)h->partials.bytes;
  }
  return FE_OK;
}

}  // namespace fe
