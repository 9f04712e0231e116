// SpMM, Y = A X for a 0/1 pattern matrix A (Section 3.3): every non-zero (i, j) adds row j
// of the dense block X to row i of Y.  X and Y are row-major n x b (Section 3.3.2).
//
// GB300 layout of A, built once per handle from the CSR (Section 3.3.1 / 3.3.3 motives: the
// paper fights branchy single-entry rows with SCSR+COO tiles and power-law load imbalance
// with work stealing; here the same two problems are solved by degree binning):
//   * tail rows (degree <= tail_max, default 128; 97% of the scale-22 R-MAT rows): grouped by
//     exact degree into 32-row slices whose column indices are stored transposed
//     ("SELL-32"): lane l of a warp owns row l of the slice and step t loads ell[t*32 + l],
//     one coalesced 128-byte load per step and no divergence or masked lane, since all 32
//     rows of a slice have the same degree;
//   * mid rows (tail_max < degree <= hub_min): one warp per row (a "task"), 32 consecutive
//     column indices per coalesced load, each lane gathering up to 32 bytes of an X row
//     (one 256-bit load when X is 32-byte aligned), partial sums combined by a
//     reduce-scatter butterfly;
//   * hub rows (degree > hub_min): split into tasks of hub_chunk non-zeros; each task writes
//     a partial row, and a second kernel adds a hub's partials in task order (deterministic,
//     no atomics).
// Tasks are ordered longest first so the block scheduler handles them like a longest-
// processing-time list; tail slices follow in the same launch.  The task rows' column
// indices are stored either as int32 or, in the packed format, as per-task gap fields that a
// warp decodes with a prefix sum (fewer bytes to stream from host memory).
// FP32 sums are compensated per lane (Kahan) before the lane tree, and hub chunks are added in
// compensated FP64, so the FP32 error bound (9 * 2^-24 * A|X| per entry) does not grow with the
// degree or depend on the signs of X.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fe_internal.cuh"
#include "vec.cuh"

namespace fe {

static_assert(sizeof(Task) == 16, "Task must be 16 bytes");
static_assert(sizeof(PTask) == 32, "PTask must be 32 bytes");

// Per (type, b, fragment width) geometry: a lane moves NE elements (<= FB bytes: 16, or 32
// with 256-bit loads when X is 32-byte aligned) per load; an X row of b elements spans C lanes
// in a warp task (P = 32 / C rows gathered per warp instruction) and C chunks in a tail lane.
template <typename T, int B, bool V32>
struct Geo {
  static constexpr int FB = V32 ? 32 : 16;
  static constexpr int ROWB = B * (int)sizeof(T);
  static constexpr int NE = ROWB <= FB ? B : FB / (int)sizeof(T);
  static constexpr int C = B / NE;
  static constexpr int P = 32 / C;
  static constexpr int UNROLL = C >= 4 ? 1 : 4 / C;
  static constexpr int LNE = NE >= 8 ? 3 : NE >= 4 ? 2 : NE >= 2 ? 1 : 0;  // log2(NE)
  // lane bits summed by the plain butterfly levels after the scatter levels (C .. 16 >> LNE)
  static constexpr int PLAIN_MASK = (16 >> LNE) >= C ? ((16 >> LNE) << 1) - C : 0;
};

struct SpmmParams {
  const int32_t* colidx;
  const uint32_t* tbits;
  const Task* tasks;
  const PTask* ptasks;
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

// Per-lane running sums.  FP32: Kahan's compensated summation (Kahan 1965; Higham, "Accuracy
// and Stability of Numerical Algorithms", 2nd ed., Thm. 4.8): c carries the rounding error of
// the last addition, so a lane's sum of m terms is within (2u + O(m u^2)) sum |x| of the exact
// sum (u = 2^-24), whatever the number of terms and their signs, instead of (m - 1) u sum |x|.
// Four FP32 adds per term; nvcc does not reassociate floating-point adds, so the correction
// survives compilation.  FP64: plain adds (m u with u = 2^-53 is already far below the FP64
// bound).  kahan_add(s, c, x) adds x; kahan_value(s, c) is the compensated sum.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
__device__ __forceinline__ void kahan_add(double& s, double&, double x) { s += x; }
__device__ __forceinline__ float kahan_value(float s, float c) { return s - c; }
__device__ __forceinline__ double kahan_value(double s, double) { return s; }

template <typename T, int B, bool V32, bool PACKED>
__device__ __forceinline__ void run_task(const SpmmParams& p, int64_t ti, const T* __restrict__ X,
                                         T* __restrict__ Y, T* __restrict__ partial, int lane) {
  using G = Geo<T, B, V32>;
  int64_t start;
  int row, len;
  int cbase = 0, w = 1;
  if constexpr (PACKED) {
    const int4 r0 = __ldg(reinterpret_cast<const int4*>(p.ptasks + ti));
    const int4 r1 = __ldg(reinterpret_cast<const int4*>(p.ptasks + ti) + 1);
    start = (int64_t)(uint32_t)r0.x | ((int64_t)r0.y << 32);  // word offset
    row = r0.z;
    len = r0.w;
    cbase = r1.x;
    w = r1.y;
  } else {
    const int4 raw = __ldg(reinterpret_cast<const int4*>(p.tasks + ti));
    start = (int64_t)(uint32_t)raw.x | ((int64_t)raw.y << 32);
    row = raw.z;
    len = raw.w;
  }
  const int chunk = lane % G::C;
  const int slot = lane / G::C;
  T acc[G::NE], cmp[G::NE];
#pragma unroll
  for (int e = 0; e < G::NE; ++e) acc[e] = cmp[e] = T(0);
  const int32_t* __restrict__ ci = p.colidx + start;
  const uint32_t* __restrict__ tb = p.tbits + start;
  const uint32_t wmask = (1u << w) - 1u;  // 1 <= w <= 31
  int carry = cbase;  // packed: the column reached by the previous round
  for (int base = 0; base < len; base += 32 * G::UNROLL) {
    int cols[G::UNROLL];
#pragma unroll
    for (int u = 0; u < G::UNROLL; ++u) {
      int k = base + u * 32 + lane;
      if constexpr (PACKED) {
        // field k of w bits, then an inclusive prefix sum of the gaps across the warp
        if (base + u * 32 < len) {
          int g = 0;
          if (k < len) {
            const int64_t bit = (int64_t)k * w;
            const int64_t wi = bit >> 5;
            g = (int)(__funnelshift_r(__ldcs(tb + wi), __ldcs(tb + wi + 1), (int)(bit & 31)) & wmask);
          }
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, g, off);
            if (lane >= off) g += y;
          }
          const int col = carry + g;
          carry = __shfl_sync(kFull, col, 31);
          cols[u] = k < len ? col : -1;
        } else {
          cols[u] = -1;
        }
      } else {
        cols[u] = k < len ? __ldcs(ci + k) : -1;
      }
    }
#pragma unroll
    for (int u = 0; u < G::UNROLL; ++u) {
#pragma unroll
      for (int g = 0; g < 32; g += G::P) {
        // rounds whose P slots all lie past the row's end are skipped (warp-uniform test)
        if (base + u * 32 + g < len) {
          int col = __shfl_sync(kFull, cols[u], g + slot);
          if (col >= 0) {
            T f[G::NE];
            ld_frag<T, G::NE>(X + (int64_t)col * B + chunk * G::NE, f);
#pragma unroll
            for (int e = 0; e < G::NE; ++e) kahan_add(acc[e], cmp[e], f[e]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < G::NE; ++e) acc[e] = kahan_value(acc[e], cmp[e]);
  // Sum the P slot partials of each chunk.  The first LNE butterfly levels (offsets 16, 8, ..)
  // also scatter the NE elements -- a lane keeps half of what it holds and adds its partner's
  // copy of that half -- so every level after them adds one value per lane.
  int ebase = 0;
#pragma unroll
  for (int lvl = 0; lvl < G::LNE; ++lvl) {
    const int h = G::NE >> (lvl + 1);
    const int off = 16 >> lvl;
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < (G::NE >> (lvl + 1)); ++i) {
      const T send = up ? acc[i] : acc[i + h];
      const T keep = up ? acc[i + h] : acc[i];
      acc[i] = keep + __shfl_xor_sync(kFull, send, off);
    }
    if (up) ebase += h;
  }
#pragma unroll
  for (int off = 16 >> G::LNE; off >= G::C; off >>= 1) acc[0] += __shfl_xor_sync(kFull, acc[0], off);
  if ((lane & G::PLAIN_MASK) == 0) {
    T* dst = ti < p.nhub_tasks ? partial + ti * B : Y + (int64_t)row * B;
    dst[chunk * G::NE + ebase] = acc[0];
  }
}

template <typename T, int B, bool V32>
__device__ __forceinline__ void run_slice(const SpmmParams& p, int64_t si, const T* __restrict__ X,
                                          T* __restrict__ Y, int lane) {
  using G = Geo<T, B, V32>;
  // bucket = last one whose first slice is <= si (buckets are non-empty, so strictly increasing)
  int lo = 0, hi = p.nbuckets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.bucket_slice_begin[mid] <= si) lo = mid;
    else hi = mid - 1;
  }
  const int bkt = lo;
  const int deg = p.bucket_deg[bkt];
  const int64_t off = p.bucket_ell_base[bkt] + (si - p.bucket_slice_begin[bkt]) * 32 * (int64_t)deg;
  const int row = __ldcs(p.slice_rows + si * 32 + lane);
  T acc[B], cmp[B];
#pragma unroll
  for (int e = 0; e < B; ++e) acc[e] = cmp[e] = T(0);
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
        for (int q = 0; q < G::NE; ++q) kahan_add(acc[ch * G::NE + q], cmp[ch * G::NE + q], f[q]);
      }
  }
  for (; t < deg; ++t) {
    int c = __ldcs(e + t * 32);
#pragma unroll
    for (int ch = 0; ch < G::C; ++ch) {
      T f[G::NE];
      ld_frag<T, G::NE>(X + (int64_t)c * B + ch * G::NE, f);
#pragma unroll
      for (int q = 0; q < G::NE; ++q) kahan_add(acc[ch * G::NE + q], cmp[ch * G::NE + q], f[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < B; ++q) acc[q] = kahan_value(acc[q], cmp[q]);
  if (row >= 0) {
    using F = FragOf<T, B>;  // stores in 16-byte pieces
#pragma unroll
    for (int ch = 0; ch < F::NCH; ++ch) st_frag<T, F::NE>(Y + (int64_t)row * B + ch * F::NE, acc + ch * F::NE);
  }
}

template <typename T, int B, bool V32, bool PACKED>
__global__ void __launch_bounds__(256) spmm_main_kernel(const SpmmParams p, const T* __restrict__ X,
                                                        T* __restrict__ Y, T* __restrict__ partial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((int64_t)blockIdx.x < p.task_ctas) {
    const int64_t ti = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    if (ti < p.ntasks) run_task<T, B, V32, PACKED>(p, ti, X, Y, partial, lane);
  } else {
    const int64_t si = ((int64_t)blockIdx.x - p.task_ctas) * kWarpsPerCta + warp;
    if (si < p.nslices) run_slice<T, B, V32>(p, si, X, Y, lane);
  }
}

// Y[hub_rows[h]] = sum of the hub's task partials in task order, in FP64 with Neumaier's
// compensation (Neumaier 1974: the TwoSum error of every add is collected separately), then
// one rounding to T: the partials add with an error of at most 2^-53 |sum| + O(k 2^-106) sum
// |partial| whatever their number k, so a hub adds one rounding of T to its chunks' errors.
template <typename T, int B>
__global__ void hub_reduce_kernel(const int32_t* __restrict__ hub_rows,
                                  const int32_t* __restrict__ hub_task_begin, int64_t nhub,
                                  const T* __restrict__ partial, T* __restrict__ Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nhub * B) return;
  const int64_t h = i / B;
  const int c = (int)(i % B);
  double s = 0.0, e = 0.0;
  for (int t = hub_task_begin[h]; t < hub_task_begin[h + 1]; ++t) {
    const double x = (double)partial[(int64_t)t * B + c];
    const double u = s + x;
    e += fabs(s) >= fabs(x) ? (s - u) + x : (x - u) + s;
    s = u;
  }
  Y[(int64_t)hub_rows[h] * B + c] = (T)(s + e);
}

// Window size for an L2 access-policy window over `bytes` of X: the device's largest window,
// the persisting set-aside (raised once per device, in this process's context, to the device's
// maximum) bounding it so that the whole window can persist.
static int l2_window_bytes(size_t bytes, size_t* win) {
  static std::mutex mu;
  static size_t maxwin[kMaxDevices], persist[kMaxDevices];
  const int dev = cur_device();
  if (dev < 0) return dev;
  std::lock_guard<std::mutex> lock(mu);
  if (maxwin[dev] == 0) {
    int mw = 0, mp = 0;
    FE_CUDA(cudaDeviceGetAttribute(&mw, cudaDevAttrMaxAccessPolicyWindowSize, dev));
    FE_CUDA(cudaDeviceGetAttribute(&mp, cudaDevAttrMaxPersistingL2CacheSize, dev));
    FE_ARG(mw > 0 && mp > 0, "spmm: this device has no L2 persistence control");
    FE_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)mp));
    maxwin[dev] = (size_t)mw;
    persist[dev] = (size_t)mp;
  }
  *win = std::min(bytes, std::min(maxwin[dev], persist[dev]));
  return FE_OK;
}

template <typename T, int B>
static int launch_spmm(const PlanView& pv, const T* X, T* Y, T* partial, cudaStream_t s) {
  SpmmParams p;
  memset(&p, 0, sizeof(p));
  p.colidx = pv.colidx;
  p.tbits = pv.tbits;
  p.tasks = reinterpret_cast<const Task*>(pv.tasks);
  p.ptasks = reinterpret_cast<const PTask*>(pv.tasks);
  p.ntasks = pv.ntasks;
  p.nhub_tasks = pv.nhub_tasks;
  p.slice_rows = pv.slice_rows;
  p.ell = pv.ell;
  p.nslices = pv.nslices;
  p.nbuckets = pv.nbuckets;
  for (int i = 0; i < pv.nbuckets; ++i) {
    p.bucket_deg[i] = pv.deg_of_bucket[i];
    p.bucket_slice_begin[i] = pv.deg_slice_begin[i];
    p.bucket_ell_base[i] = pv.deg_ell_base[i];
  }
  p.bucket_slice_begin[pv.nbuckets] = (int32_t)pv.nslices;
  p.task_ctas = ceil_div(pv.ntasks, kWarpsPerCta);
  const int64_t ctas = p.task_ctas + ceil_div(pv.nslices, kWarpsPerCta);
  if (ctas > 0) {
    // 256-bit gathers when an X row spans at least 32 bytes and X is 32-byte aligned
    bool v32 = false;
    if constexpr (B * sizeof(T) >= 32) v32 = ((uintptr_t)X % 32) == 0;
    void (*kern)(const SpmmParams, const T*, T*, T*) = nullptr;
    if (v32) {
      if constexpr (B * sizeof(T) >= 32)
        kern = pv.packed ? spmm_main_kernel<T, B, true, true> : spmm_main_kernel<T, B, true, false>;
    } else {
      kern = pv.packed ? spmm_main_kernel<T, B, false, true> : spmm_main_kernel<T, B, false, false>;
    }
    if (pv.l2_persist) {
      // L2 access-policy window on X: its lines are kept (persisting) while the streamed index
      // arrays pass through as streaming accesses (Section 3.3.3's cache-resident dense tiles,
      // with the GPU's L2 as the cache)
      size_t win = 0;
      FE_TRY(l2_window_bytes((size_t)pv.x_rows * B * sizeof(T), &win));
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
      attr[0].val.accessPolicyWindow.base_ptr = const_cast<T*>(X);
      attr[0].val.accessPolicyWindow.num_bytes = win;
      attr[0].val.accessPolicyWindow.hitRatio = 1.0f;
      attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
      attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)ctas);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      FE_CUDA(cudaLaunchKernelEx(&cfg, kern, p, X, Y, partial));
    } else {
      kern<<<(unsigned)ctas, 256, 0, s>>>(p, X, Y, partial);
    }
    count_launch();
    FE_CUDA(cudaGetLastError());
  }
  if (pv.nhub > 0) {
    const int64_t th = pv.nhub * B;
    hub_reduce_kernel<T, B><<<(unsigned)ceil_div(th, 256), 256, 0, s>>>(
        pv.hub_rows, pv.hub_task_begin, pv.nhub, partial, Y);
    count_launch();
    FE_CUDA(cudaGetLastError());
  }
  return FE_OK;
}

PlanView resident_view(fe_csr h) {
  const fe_spmm_plan& pl = h->plan;
  PlanView v;
  memset(&v, 0, sizeof(v));
  v.colidx = h->d_colidx;
  v.tbits = pl.d_tbits;
  v.packed = pl.packed;
  v.tasks = pl.d_tasks;
  v.ntasks = pl.ntasks;
  v.nhub_tasks = pl.nhub_tasks;
  v.slice_rows = pl.d_slice_rows;
  v.ell = pl.d_ell;
  v.nslices = pl.nslices;
  v.nbuckets = pl.nbuckets;
  for (int i = 0; i < pl.nbuckets; ++i) {
    v.deg_of_bucket[i] = pl.deg_of_bucket[i];
    v.deg_slice_begin[i] = pl.deg_slice_begin[i];
    v.deg_ell_base[i] = pl.deg_ell_base[i];
  }
  v.hub_rows = pl.d_hub_rows;
  v.hub_task_begin = pl.d_hub_task_begin;
  v.nhub = pl.nhub;
  v.x_rows = h->ncols;
  v.l2_persist = pl.l2_persist;
  return v;
}

int spmm_view(const PlanView& v, const void* X, void* Y, void* partial, int b, fe_dtype dt,
              cudaStream_t s) {
  if (dt == FE_F32) {
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    float* pa = static_cast<float*>(partial);
    switch (b) {
      case 1: return launch_spmm<float, 1>(v, x, y, pa, s);
      case 2: return launch_spmm<float, 2>(v, x, y, pa, s);
      case 4: return launch_spmm<float, 4>(v, x, y, pa, s);
      case 8: return launch_spmm<float, 8>(v, x, y, pa, s);
      case 16: return launch_spmm<float, 16>(v, x, y, pa, s);
    }
  } else {
    const double* x = static_cast<const double*>(X);
    double* y = static_cast<double*>(Y);
    double* pa = static_cast<double*>(partial);
    switch (b) {
      case 1: return launch_spmm<double, 1>(v, x, y, pa, s);
      case 2: return launch_spmm<double, 2>(v, x, y, pa, s);
      case 4: return launch_spmm<double, 4>(v, x, y, pa, s);
      case 8: return launch_spmm<double, 8>(v, x, y, pa, s);
      case 16: return launch_spmm<double, 16>(v, x, y, pa, s);
    }
  }
  return set_error(FE_ERR_INVALID, "spmm: unsupported b = %d", b);
}

int spmm_resident(fe_csr h, const void* X, void* Y, int b, fe_dtype dt, cudaStream_t s) {
  return spmm_view(resident_view(h), X, Y, h->partials.p, b, dt, s);
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

// Plan of rows [r0, r1): task starts are offsets into hp.tcol, the column indices of the
// panel's task rows only (tail rows are read from the ELL slices); row ids are global.
static int bit_length(uint32_t x) { return x == 0 ? 0 : 32 - __builtin_clz(x); }

size_t plan_row_index_bytes(const int32_t* cols, int64_t d, int tail_max, int hub_chunk, bool packed) {
  if (d <= tail_max || !packed) return 4 * (size_t)d;
  // packed: every chunk of hub_chunk entries is a segment of one gap width, word-aligned
  std::vector<int32_t> sorted;
  const int32_t* c = cols;
  if (!std::is_sorted(cols, cols + d)) {
    sorted.assign(cols, cols + d);
    std::sort(sorted.begin(), sorted.end());
    c = sorted.data();
  }
  size_t bytes = 0;
  for (int64_t s0 = 0; s0 < d; s0 += hub_chunk) {
    const int64_t s1 = std::min<int64_t>(d, s0 + hub_chunk);
    int w = 1;
    for (int64_t k = s0 + 1; k < s1; ++k) w = std::max(w, bit_length((uint32_t)(c[k] - c[k - 1])));
    bytes += 4 * (size_t)ceil_div((s1 - s0) * w, 32) + 16;  // + the larger task record
  }
  return bytes;
}

// Packed index format: each task's sorted columns become gap fields of the task's width w
// (g_0 = 0, g_k = c_k - c_{k-1}) in a word-aligned segment of the bit stream, so that tasks can
// be encoded in parallel; two zero words pad the end (the decoder reads a two-word window).
static void pack_tasks(HostPlan& hp) {
  const int64_t nt = hp.ntasks;
  hp.ptasks.resize(nt);
  std::vector<int64_t> words(nt + 1, 0);
  #pragma omp parallel for schedule(dynamic, 256)
  for (int64_t t = 0; t < nt; ++t) {
    const Task& tk = hp.tasks[t];
    const int32_t* c = hp.tcol.data() + tk.start;
    int w = 1;
    for (int k = 1; k < tk.len; ++k) w = std::max(w, bit_length((uint32_t)(c[k] - c[k - 1])));
    hp.ptasks[t] = PTask{0, tk.row, tk.len, c[0], w, 0, 0};
    words[t + 1] = ceil_div((int64_t)tk.len * w, 32);
  }
  for (int64_t t = 0; t < nt; ++t) words[t + 1] += words[t];
  hp.tbits.assign(words[nt] + 2, 0u);
  #pragma omp parallel for schedule(dynamic, 256)
  for (int64_t t = 0; t < nt; ++t) {
    PTask& pt = hp.ptasks[t];
    pt.woff = words[t];
    const int32_t* c = hp.tcol.data() + hp.tasks[t].start;
    uint32_t* out = hp.tbits.data() + words[t];
    const int w = pt.w;
    for (int k = 1; k < pt.len; ++k) {
      const uint32_t g = (uint32_t)(c[k] - c[k - 1]);
      const int64_t bit = (int64_t)k * w;
      const int64_t wi = bit >> 5;
      const int sh = (int)(bit & 31);
      out[wi] |= g << sh;
      if (sh + w > 32) out[wi + 1] |= g >> (32 - sh);
    }
  }
  hp.tcol.clear();
  hp.tcol.shrink_to_fit();
  hp.tasks.clear();
  hp.tasks.shrink_to_fit();
  hp.packed = true;
}

int build_host_plan(const int64_t* rowptr, const int32_t* colidx, int64_t r0, int64_t r1,
                    int tail_max, int hub_min, int hub_chunk, bool packed, HostPlan& hp) {
  hp = HostPlan();
  std::vector<int64_t> tail_cnt(tail_max + 1, 0);
  std::vector<int64_t> mid_cnt(hub_min + 1, 0);
  int64_t nhub = 0, nhub_tasks = 0;
  for (int64_t i = r0; i < r1; ++i) {
    const int64_t d = rowptr[i + 1] - rowptr[i];
    hp.max_degree = std::max(hp.max_degree, d);
    if (d <= tail_max) tail_cnt[d]++;
    else if (d <= hub_min) mid_cnt[d]++;
    else { nhub++; nhub_tasks += ceil_div(d, hub_chunk); }
  }
  hp.rows_empty = tail_cnt[0];
  for (int d = 1; d <= tail_max; ++d) hp.rows_tail += tail_cnt[d];
  for (int d = tail_max + 1; d <= hub_min; ++d) hp.rows_mid += mid_cnt[d];
  hp.rows_hub = nhub;
  FE_ARG(nhub_tasks < INT32_MAX, "spmm plan: too many hub tasks");
  // tail slices: buckets by degree, descending, empty buckets dropped
  int64_t nslices = 0, ell_total = 0;
  std::vector<int> bucket_of_deg(tail_max + 1, -1);
  for (int d = tail_max; d >= 0; --d) {
    if (tail_cnt[d] == 0) continue;
    const int bk = hp.nbuckets++;
    bucket_of_deg[d] = bk;
    hp.deg_of_bucket[bk] = d;
    hp.deg_slice_begin[bk] = (int32_t)nslices;
    hp.deg_ell_base[bk] = ell_total;
    const int64_t sl = ceil_div(tail_cnt[d], 32);
    nslices += sl;
    ell_total += sl * 32 * d;
  }
  FE_ARG(nslices < INT32_MAX, "spmm plan: too many tail slices");
  hp.nslices = nslices;
  hp.slice_rows.assign(nslices * 32, -1);
  std::vector<int64_t> cursor(tail_max + 1, 0);
  for (int d = 0; d <= tail_max; ++d)
    if (bucket_of_deg[d] >= 0) cursor[d] = (int64_t)hp.deg_slice_begin[bucket_of_deg[d]] * 32;
  // tasks: hub chunks first, then mid rows by degree descending (stable in row order)
  std::vector<int64_t> mid_pos(hub_min + 2, 0);
  {
    int64_t acc = nhub_tasks;
    for (int d = hub_min; d > tail_max; --d) { mid_pos[d] = acc; acc += mid_cnt[d]; }
  }
  hp.ntasks = nhub_tasks + hp.rows_mid;
  hp.nhub_tasks = nhub_tasks;
  hp.nhub = nhub;
  hp.tasks.resize(hp.ntasks);
  hp.hub_rows.resize(nhub);
  hp.hub_task_begin.resize(nhub + 1);
  int64_t ht = 0, hi = 0, tpos = 0;
  {
    int64_t tnnz = 0;
    for (int64_t i = r0; i < r1; ++i) {
      const int64_t d = rowptr[i + 1] - rowptr[i];
      if (d > tail_max) tnnz += d;
    }
    hp.tcol.resize(tnnz > 0 ? tnnz : 1);
  }
  for (int64_t i = r0; i < r1; ++i) {
    const int64_t d = rowptr[i + 1] - rowptr[i];
    if (d <= tail_max) {
      hp.slice_rows[cursor[d]++] = (int32_t)i;
      continue;
    }
    memcpy(hp.tcol.data() + tpos, colidx + rowptr[i], sizeof(int32_t) * (size_t)d);
    if (packed && !std::is_sorted(hp.tcol.data() + tpos, hp.tcol.data() + tpos + d))
      std::sort(hp.tcol.data() + tpos, hp.tcol.data() + tpos + d);
    if (d <= hub_min) {
      hp.tasks[mid_pos[d]++] = Task{tpos, (int32_t)i, (int32_t)d};
    } else {
      hp.hub_rows[hi] = (int32_t)i;
      hp.hub_task_begin[hi] = (int32_t)ht;
      for (int64_t c = 0; c < d; c += hub_chunk)
        hp.tasks[ht++] = Task{tpos + c, (int32_t)i, (int32_t)std::min<int64_t>(hub_chunk, d - c)};
      ++hi;
    }
    tpos += d;
  }
  hp.tcol_total = tpos;
  hp.hub_task_begin[nhub] = (int32_t)ht;
  // ELL fill (transposed per slice; padding lanes read column 0 and are not written)
  hp.ell.assign(ell_total > 0 ? ell_total : 1, 0);
  for (int bk = 0; bk < hp.nbuckets; ++bk) {
    const int d = hp.deg_of_bucket[bk];
    if (d == 0) continue;
    const int64_t s0 = hp.deg_slice_begin[bk];
    const int64_t s1 = (bk + 1 < hp.nbuckets) ? hp.deg_slice_begin[bk + 1] : nslices;
    int32_t* ell = hp.ell.data();
    const int32_t* srows = hp.slice_rows.data();
    const int64_t ebase = hp.deg_ell_base[bk];
    #pragma omp parallel for schedule(static)
    for (int64_t sl = s0; sl < s1; ++sl) {
      int32_t* e = ell + ebase + (sl - s0) * 32 * d;
      for (int lane = 0; lane < 32; ++lane) {
        const int32_t r = srows[sl * 32 + lane];
        for (int t = 0; t < d; ++t) e[t * 32 + lane] = r >= 0 ? colidx[rowptr[r] + t] : 0;
      }
    }
  }
  hp.ell_total = ell_total;
  if (packed) pack_tasks(hp);
  return FE_OK;
}

int spmm_build_plan(fe_csr h, const int64_t* rowptr, const int32_t* colidx_raw, int tail_max,
                    int hub_min, int hub_chunk, bool packed) {
  const int64_t n = h->n;
  const int32_t* colidx = colidx_raw;
  fe_spmm_plan& pl = h->plan;
  pl.tail_max = tail_max;
  pl.hub_min = hub_min;
  pl.hub_chunk = hub_chunk;
  HostPlan hp;
  FE_TRY(build_host_plan(rowptr, colidx, 0, n, tail_max, hub_min, hub_chunk, packed, hp));
  pl.packed = packed ? 1 : 0;
  h->max_degree = hp.max_degree;
  h->rows_empty = hp.rows_empty;
  h->rows_tail = hp.rows_tail;
  h->rows_mid = hp.rows_mid;
  h->rows_hub = hp.rows_hub;
  pl.nbuckets = hp.nbuckets;
  for (int i = 0; i < hp.nbuckets; ++i) {
    pl.deg_of_bucket[i] = hp.deg_of_bucket[i];
    pl.deg_slice_begin[i] = hp.deg_slice_begin[i];
    pl.deg_ell_base[i] = hp.deg_ell_base[i];
  }
  pl.nslices = hp.nslices;
  pl.ntasks = hp.ntasks;
  pl.nhub_tasks = hp.nhub_tasks;
  pl.nhub = hp.nhub;
  if (packed) {
    FE_TRY(dev_upload(h, (void**)&pl.d_tbits, hp.tbits.data(), sizeof(uint32_t) * hp.tbits.size()));
    FE_TRY(dev_upload(h, &pl.d_tasks, hp.ptasks.data(), sizeof(PTask) * hp.ntasks));
    pl.index_bytes = (int64_t)(sizeof(uint32_t) * hp.tbits.size() + sizeof(int32_t) * hp.ell_total);
  } else {
    FE_TRY(dev_upload(h, (void**)&h->d_colidx, hp.tcol.data(), sizeof(int32_t) * hp.tcol_total));
    FE_TRY(dev_upload(h, &pl.d_tasks, hp.tasks.data(), sizeof(Task) * hp.ntasks));
    pl.index_bytes = (int64_t)(sizeof(int32_t) * (hp.tcol_total + hp.ell_total));
  }
  FE_TRY(dev_upload(h, (void**)&pl.d_slice_rows, hp.slice_rows.data(), sizeof(int32_t) * hp.slice_rows.size()));
  FE_TRY(dev_upload(h, (void**)&pl.d_ell, hp.ell.data(), sizeof(int32_t) * hp.ell_total));
  FE_TRY(dev_upload(h, (void**)&pl.d_hub_rows, hp.hub_rows.data(), sizeof(int32_t) * hp.nhub));
  FE_TRY(dev_upload(h, (void**)&pl.d_hub_task_begin, hp.hub_task_begin.data(), sizeof(int32_t) * (hp.nhub + 1)));
  if (hp.nhub_tasks > 0) {
    FE_TRY(h->partials.alloc(sizeof(double) * 16 * hp.nhub_tasks));
    h->device_bytes += (int64_t)h->partials.bytes;
  }
  return FE_OK;
}

}  // namespace fe
