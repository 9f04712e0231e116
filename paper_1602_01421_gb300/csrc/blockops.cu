// Dense tall-and-skinny block operations of Table 1 on row-major n x b blocks.
//
//   gram     MvTransMv ("op3"): G = alpha V^T W.  Two phases as in Section 3.4.2 (each CTA
//            reduces its row ranges to a small partial matrix, then one pass adds the partials
//            in a fixed order -- deterministic, no atomics).  Inside a CTA a range of W rows is
//            staged in shared memory once; each warp owns up to two (block j, column group)
//            output tiles for the whole launch, sweeps every range with lane = row (four row
//            loads in flight per lane) and reduces across lanes once at the end, so every V
//            element is read once, coalesced.  The grid is as many CTAs as fit on the GPU.
//   update   MvTimesMatAddMv ("op1") fused with MvScale1/2: W = beta W M + alpha V C; one
//            thread per row, C and M in shared memory.
//   combine  V_out = V Y (restart and Ritz vectors: n x m times m x k).
//   random   MvRandom with a counter-based generator.
// FP32 blocks use FP32 products and per-thread sums; Gram partials are combined in FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fe_internal.cuh"
#include "vec.cuh"

namespace fe {

constexpr unsigned kFullMask = 0xffffffffu;

// ---------------------------------------------------------------- scratch pools
constexpr int kScratchSlots = 32;
struct ScratchPool {
  DevBuf bufs[kScratchSlots];
};
// One pool per (host thread, device), created on first use and kept until the thread exits,
// so a thread that switches devices keeps every device's buffers instead of reallocating them.
struct ThreadPools {
  ScratchPool* p[kMaxDevices] = {};
  ~ThreadPools() {
    for (ScratchPool* q : p) delete q;
  }
};
static thread_local ThreadPools t_pools;

static ScratchPool* pool() {
  const int dev = cur_device();
  if (dev < 0) return nullptr;
  if (!t_pools.p[dev]) t_pools.p[dev] = new ScratchPool();
  return t_pools.p[dev];
}

double* small_scratch(int slot, size_t count) {
  if (slot < 0 || slot >= kScratchSlots) {
    set_error(FE_ERR_INVALID, "internal: scratch slot %d out of range", slot);
    return nullptr;
  }
  ScratchPool* pl = pool();
  if (!pl) return nullptr;
  DevBuf& b = pl->bufs[slot];
  if (b.alloc(count * sizeof(double)) != FE_OK) return nullptr;
  return b.as<double>();
}

// ---------------------------------------------------------------- row loaders for BlockSets
template <typename T, int BV>
__device__ __forceinline__ void load_vrow(const T* __restrict__ base, int ld, int64_t r, T* v) {
  if (ld == BV) {
    ld_row<T, BV>(base + r * BV, v);
  } else {
#pragma unroll
    for (int p = 0; p < BV; ++p) v[p] = base[r * ld + p];
  }
}

// ---------------------------------------------------------------- gram
// Rows [r, r + rows) of tile (j, q0) of V_j^T W from the staged W rows sW (lane = row, four
// row loads in flight per lane when the block is narrow).  Products and sums in TC (T, or
// float for FP64 blocks when only a first-pass estimate is wanted).
template <typename T, typename TC, int BV, int NQ>
__device__ __forceinline__ void gram_tile_rows(const T* __restrict__ vb, int ldv, int64_t r0, int rows,
                                               const TC* sW, int bw, int q0, int lane, TC (&acc)[BV][NQ]) {
  constexpr int U = BV >= 16 ? 1 : (BV >= 8 ? 2 : 4);
  int r = lane;
  for (; r + 32 * (U - 1) < rows; r += 32 * U) {
    T v[U][BV];
#pragma unroll
    for (int u = 0; u < U; ++u) load_vrow<T, BV>(vb, ldv, r0 + r + 32 * u, v[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const TC* w = sW + (r + 32 * u) * bw + q0;
#pragma unroll
      for (int p = 0; p < BV; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[p][q] = fma(to_arith<TC>(v[u][p]), w[q], acc[p][q]);
    }
  }
  for (; r < rows; r += 32) {
    T v[BV];
    load_vrow<T, BV>(vb, ldv, r0 + r, v);
    const TC* w = sW + r * bw + q0;
#pragma unroll
    for (int p = 0; p < BV; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[p][q] = fma(to_arith<TC>(v[p]), w[q], acc[p][q]);
  }
}

template <typename T, int BV, int NQ>
__device__ __forceinline__ void gram_tile_flush(T (&acc)[BV][NQ], double* sP, int row0, int bw, int q0,
                                                int lane) {
#pragma unroll
  for (int p = 0; p < BV; ++p)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double a = (double)acc[p][q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(kFullMask, a, off);
      if (lane == 0) sP[(row0 + p) * bw + q0 + q] += a;
      acc[p][q] = T(0);
    }
}

// Output tiles are (block j, NQ columns of W).  TPW > 0: warp w owns tiles w + 8t (t < TPW) for
// the whole launch and reduces its accumulators across lanes once, at the end; TPW == 0 (more
// tiles than that): tiles are dealt out per staged range and reduced per range.
template <typename T, int BV, int NQ, int TPW, typename TC = T>
__global__ void __launch_bounds__(256) gram_kernel(const BlockSet V, const T* __restrict__ W,
                                                   int ldw, int bw, int64_t n, int R,
                                                   double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* sW = reinterpret_cast<TC*>(smem_raw);
  double* sP = reinterpret_cast<double*>(smem_raw + (((size_t)R * bw * sizeof(TC) + 15) & ~(size_t)15));
  const int nout = V.nv * BV * bw;
  for (int e = threadIdx.x; e < nout; e += blockDim.x) sP[e] = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarps = 8;
  const int qtiles = bw / NQ;
  const int ntiles = V.nv * qtiles;
  constexpr int NT = TPW > 0 ? TPW : 1;
  TC acc[NT][BV][NQ];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int p = 0; p < BV; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[t][p][q] = TC(0);
  constexpr bool kSame = sizeof(T) == sizeof(TC);
  const bool vec = kSame && ldw == bw && ((size_t)bw * sizeof(T)) % 16 == 0 &&
                   (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < n; r0 += (int64_t)gridDim.x * R) {
    const int rows = (int)min((int64_t)R, n - r0);
    __syncthreads();
    if (vec) {
      const int4* src = reinterpret_cast<const int4*>(W + r0 * bw);
      int4* dst = reinterpret_cast<int4*>(sW);
      const int n16 = (int)(((size_t)rows * bw * sizeof(T)) / 16);
      for (int e = threadIdx.x; e < n16; e += blockDim.x) dst[e] = src[e];
    } else {
      for (int rr = threadIdx.x; rr < rows; rr += blockDim.x)
        for (int q = 0; q < bw; ++q) sW[rr * bw + q] = to_arith<TC>(W[(r0 + rr) * ldw + q]);
    }
    __syncthreads();
    if (TPW > 0) {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int tile = warp + kWarps * t;
        if (tile < ntiles) {
          const int j = tile / qtiles, q0 = (tile % qtiles) * NQ;
          gram_tile_rows<T, TC, BV, NQ>(reinterpret_cast<const T*>(V.blk[j]), V.ld, r0, rows, sW, bw, q0, lane, acc[t]);
        }
      }
    } else {
      for (int tile = warp; tile < ntiles; tile += kWarps) {
        const int j = tile / qtiles, q0 = (tile % qtiles) * NQ;
        gram_tile_rows<T, TC, BV, NQ>(reinterpret_cast<const T*>(V.blk[j]), V.ld, r0, rows, sW, bw, q0, lane, acc[0]);
        gram_tile_flush<TC, BV, NQ>(acc[0], sP, j * BV, bw, q0, lane);
      }
    }
  }
  if (TPW > 0) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int tile = warp + kWarps * t;
      if (tile < ntiles) {
        const int j = tile / qtiles, q0 = (tile % qtiles) * NQ;
        gram_tile_flush<TC, BV, NQ>(acc[t], sP, j * BV, bw, q0, lane);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nout; e += blockDim.x) partial[(int64_t)blockIdx.x * nout + e] = sP[e];
}

// G[e] = alpha * sum_c partial[c * nout + e]: one warp per output; lane l adds partials
// l, l + 32, ... in order, then a fixed xor tree -- the same order on every call.
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nctas, int nout,
                                   double alpha, double* __restrict__ G) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= nout) return;
  double s = 0.0;
#pragma unroll 8
  for (int c = lane; c < nctas; c += 32) s += partial[(int64_t)c * nout + e];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFullMask, s, off);
  if (lane == 0) G[e] = alpha * s;
}

static int launch_gram_reduce(const double* part, int nctas, int nout, double alpha, double* G,
                              cudaStream_t s) {
  gram_reduce_kernel<<<(unsigned)ceil_div(nout, 8), 256, 0, s>>>(part, nctas, nout, alpha, G);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int gram_reduce(const double* partial, int nctas, int nout, double alpha, double* G, cudaStream_t s) {
  return launch_gram_reduce(partial, nctas, nout, alpha, G, s);
}

// Launches gram_kernel<T, BV, NQ, TPW> with as many CTAs as fit on the GPU at once (at most one
// staged range each per pass), then the partial reduction.  scratch == nullptr: partials in
// the pool's slot 0; otherwise in scratch (capacity doubles), the grid shrunk to fit.
template <typename T, int BV, int NQ, int TPW, typename TC = T>
static int launch_gram_tpw(const BlockSet& V, int64_t n, const T* W, int bw, int ldw, double alpha,
                           double* G, double* scratch, size_t capacity, cudaStream_t s) {
  const int nout = V.nv * BV * bw;
  int R = (int)(16384 / ((size_t)bw * sizeof(TC)));
  R = std::max(32, R - R % 32);
  const size_t smem = (((size_t)R * bw * sizeof(TC) + 15) & ~(size_t)15) + (size_t)nout * sizeof(double);
  FE_ARG(smem <= 200 * 1024, "gram: output too large (%d entries)", nout);
  static KernelSetup ks;
  const void* fn = reinterpret_cast<const void*>(gram_kernel<T, BV, NQ, TPW, TC>);
  FE_TRY(kernel_configure(ks, fn, 200 * 1024));
  int per_sm = 0;
  FE_TRY(kernel_occupancy(ks, fn, 256, smem, 0, &per_sm));
  int64_t nctas = std::min<int64_t>(ceil_div(n, R), (int64_t)per_sm * num_sms());
  nctas = std::max<int64_t>(nctas, 1);
  double* part = scratch;
  if (!part) {
    part = small_scratch(0, (size_t)nctas * nout);
    if (!part) return FE_ERR_OOM;
  } else {
    nctas = std::min<int64_t>(nctas, (int64_t)(capacity / (size_t)nout));
    FE_ARG(nctas >= 1, "gram: scratch of %zu doubles cannot hold %d outputs", capacity, nout);
  }
  gram_kernel<T, BV, NQ, TPW, TC><<<(unsigned)nctas, 256, smem, s>>>(V, W, ldw, bw, n, R, part);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return launch_gram_reduce(part, (int)nctas, nout, alpha, G, s);
}

// Persistent accumulators when a warp's tiles fit in 32 32-bit registers.
template <typename T, int BV, int NQ, typename TC = T>
static int launch_gram_any(const BlockSet& V, int64_t n, const T* W, int bw, int ldw, double alpha,
                           double* G, double* scratch, size_t capacity, cudaStream_t s) {
  constexpr int kRegsPerTile = BV * NQ * (int)(sizeof(TC) / 4);
  const int ntiles = V.nv * (bw / NQ);
  if (ntiles <= 8 && kRegsPerTile <= 32)
    return launch_gram_tpw<T, BV, NQ, (kRegsPerTile <= 32 ? 1 : 0), TC>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
  if (ntiles <= 16 && 2 * kRegsPerTile <= 32)
    return launch_gram_tpw<T, BV, NQ, (2 * kRegsPerTile <= 32 ? 2 : 0), TC>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
  return launch_gram_tpw<T, BV, NQ, 0, TC>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
}

template <typename T, int BV, int NQ>
static int launch_gram(const BlockSet& V, int64_t n, const T* W, int bw, int ldw, double alpha,
                       double* G, cudaStream_t s) {
  return launch_gram_any<T, BV, NQ>(V, n, W, bw, ldw, alpha, G, nullptr, 0, s);
}

template <typename T, int BV>
static int gram_bv(const BlockSet& V, int64_t n, const T* W, int bw, int ldw, double alpha,
                   double* G, cudaStream_t s) {
  constexpr int QMAX = 32 / BV >= 16 ? 16 : 32 / BV;
  const int nq = std::min(bw, QMAX);
  switch (nq) {
    case 1: return launch_gram<T, BV, 1>(V, n, W, bw, ldw, alpha, G, s);
    case 2: return launch_gram<T, BV, (QMAX >= 2 ? 2 : 1)>(V, n, W, bw, ldw, alpha, G, s);
    case 4: return launch_gram<T, BV, (QMAX >= 4 ? 4 : 1)>(V, n, W, bw, ldw, alpha, G, s);
    case 8: return launch_gram<T, BV, (QMAX >= 8 ? 8 : 1)>(V, n, W, bw, ldw, alpha, G, s);
    case 16: return launch_gram<T, BV, (QMAX >= 16 ? 16 : 1)>(V, n, W, bw, ldw, alpha, G, s);
  }
  return set_error(FE_ERR_INVALID, "gram: bad bw %d", bw);
}

int gram(const BlockSet& V, int64_t n, const void* W, int bw, int ldw, fe_dtype dt, double alpha,
         double* G, cudaStream_t s, int engine) {
  FE_ARG(V.nv >= 1 && V.nv <= kMaxBlocks, "gram: nv = %d out of range", V.nv);
  FE_ARG(is_pow2_le16(bw), "gram: bw = %d", bw);
  FE_ARG(engine == FE_ENGINE_AUTO || engine == FE_ENGINE_FMA || engine == FE_ENGINE_TC,
         "gram: engine = %d", engine);
  // AUTO takes the split-product Gram where it is measured faster than the FP64 FMA kernels on
  // this part: V with at least 16 columns (n = 2^22, 36 x 4: 0.97 against 1.55 ms; 4 x 4: 0.38
  // against 0.31 ms)
  if (engine != FE_ENGINE_FMA && dt == FE_F64) {
    const bool ok = tc_gram_supported(V, bw, ldw, dt);
    if (ok && (engine == FE_ENGINE_TC || V.nv * V.bv >= 16))
      return tc_gram(V, n, static_cast<const double*>(W), bw, alpha, G, s);
    FE_ARG(ok || engine == FE_ENGINE_AUTO,
           "gram: the tensor-core engine takes FP64 V with nv*bv <= 36 and bw in {1, 2, 4, 8}");
  }
  FE_ARG(engine != FE_ENGINE_TC, "gram: the tensor-core engine takes FP64 blocks only");
  if (dt == FE_F32) {
    const float* w = static_cast<const float*>(W);
    switch (V.bv) {
      case 1: return gram_bv<float, 1>(V, n, w, bw, ldw, alpha, G, s);
      case 2: return gram_bv<float, 2>(V, n, w, bw, ldw, alpha, G, s);
      case 4: return gram_bv<float, 4>(V, n, w, bw, ldw, alpha, G, s);
      case 8: return gram_bv<float, 8>(V, n, w, bw, ldw, alpha, G, s);
      case 16: return gram_bv<float, 16>(V, n, w, bw, ldw, alpha, G, s);
    }
  } else {
    const double* w = static_cast<const double*>(W);
    switch (V.bv) {
      case 1: return gram_bv<double, 1>(V, n, w, bw, ldw, alpha, G, s);
      case 2: return gram_bv<double, 2>(V, n, w, bw, ldw, alpha, G, s);
      case 4: return gram_bv<double, 4>(V, n, w, bw, ldw, alpha, G, s);
      case 8: return gram_bv<double, 8>(V, n, w, bw, ldw, alpha, G, s);
      case 16: return gram_bv<double, 16>(V, n, w, bw, ldw, alpha, G, s);
    }
  }
  return set_error(FE_ERR_INVALID, "gram: bv = %d not in {1,2,4,8,16}", V.bv);
}

// G = alpha V^T W for FP64 blocks with FP32 products and per-lane FP32 sums (partials combined in
// FP64): an estimate with about 1e-6 relative error at HBM speed instead of the FP64 rate.  Only
// for first-pass Gram-Schmidt coefficients, which a second FP64 pass corrects.  V blocks and W
// are n x b with ld b.
int gram_f32_arith(const BlockSet& V, int64_t n, const double* W, int b, double alpha, double* G,
                   cudaStream_t s) {
  FE_ARG(V.nv >= 1 && V.nv <= kMaxBlocks, "gram: nv = %d out of range", V.nv);
  FE_ARG(V.bv == b, "gram: block width %d != %d", V.bv, b);
  switch (b) {
    case 1: return launch_gram_any<double, 1, 1, float>(V, n, W, b, b, alpha, G, nullptr, 0, s);
    case 2: return launch_gram_any<double, 2, 2, float>(V, n, W, b, b, alpha, G, nullptr, 0, s);
    case 4: return launch_gram_any<double, 4, 4, float>(V, n, W, b, b, alpha, G, nullptr, 0, s);
    case 8: return launch_gram_any<double, 8, 4, float>(V, n, W, b, b, alpha, G, nullptr, 0, s);
    case 16: return launch_gram_any<double, 16, 2, float>(V, n, W, b, b, alpha, G, nullptr, 0, s);
  }
  return set_error(FE_ERR_INVALID, "gram: b = %d not in {1,2,4,8,16}", b);
}

// ---------------------------------------------------------------- update
// W[r] = beta * (W[r] M) + alpha * sum_j V_j[r] C_j.  skip != null and *skip != 0 -> no-op.
template <typename T, int BV, int BW>
__global__ void __launch_bounds__(256) update_kernel(const BlockSet V, const double* __restrict__ C,
                                                     double alpha, double beta,
                                                     const double* __restrict__ M,
                                                     T* __restrict__ W, int ldw, int64_t n,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sC = reinterpret_cast<T*>(smem_raw);
  const int k = V.nv * BV;
  T* sM = sC + (size_t)k * BW;
  for (int e = threadIdx.x; e < k * BW; e += blockDim.x) sC[e] = (T)(alpha * C[e]);
  if (M)
    for (int e = threadIdx.x; e < BW * BW; e += blockDim.x) sM[e] = (T)(beta * M[e]);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    T acc[BW];
    if (beta == 0.0) {
#pragma unroll
      for (int q = 0; q < BW; ++q) acc[q] = T(0);
    } else {
      T w[BW];
      if (ldw == BW) {
        ld_row_rw<T, BW>(W + r * BW, w);
      } else {
#pragma unroll
        for (int q = 0; q < BW; ++q) w[q] = W[r * ldw + q];
      }
      if (M) {
#pragma unroll
        for (int q = 0; q < BW; ++q) {
          T a = T(0);
#pragma unroll
          for (int p = 0; p < BW; ++p) a = fma(w[p], sM[p * BW + q], a);
          acc[q] = a;
        }
      } else {
#pragma unroll
        for (int q = 0; q < BW; ++q) acc[q] = (T)beta * w[q];
      }
    }
    for (int j = 0; j < V.nv; ++j) {
      T v[BV];
      load_vrow<T, BV>(reinterpret_cast<const T*>(V.blk[j]), V.ld, r, v);
      const T* c = sC + j * BV * BW;
#pragma unroll
      for (int p = 0; p < BV; ++p)
#pragma unroll
        for (int q = 0; q < BW; ++q) acc[q] = fma(v[p], c[p * BW + q], acc[q]);
    }
    if (ldw == BW) {
      st_row<T, BW>(W + r * BW, acc);
    } else {
#pragma unroll
      for (int q = 0; q < BW; ++q) W[r * ldw + q] = acc[q];
    }
  }
}

template <typename T, int BV, int BW>
static int launch_update(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                         const double* M, T* W, int ldw, const int* skip, cudaStream_t s) {
  const size_t smem = ((size_t)V.nv * BV * BW + (size_t)BW * BW) * sizeof(T);
  FE_ARG(smem <= 200 * 1024, "update: coefficient matrix too large");
  static KernelSetup ks;
  FE_TRY(kernel_configure(ks, reinterpret_cast<const void*>(update_kernel<T, BV, BW>), 200 * 1024));
  int ctas = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
  ctas = std::max(ctas, 1);
  update_kernel<T, BV, BW><<<ctas, 256, smem, s>>>(V, C, alpha, beta, M, W, ldw, n, skip);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

template <typename T, int BV>
static int update_bv(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                     const double* M, T* W, int bw, int ldw, const int* skip, cudaStream_t s) {
  switch (bw) {
    case 1: return launch_update<T, BV, 1>(V, n, C, alpha, beta, M, W, ldw, skip, s);
    case 2: return launch_update<T, BV, 2>(V, n, C, alpha, beta, M, W, ldw, skip, s);
    case 4: return launch_update<T, BV, 4>(V, n, C, alpha, beta, M, W, ldw, skip, s);
    case 8: return launch_update<T, BV, 8>(V, n, C, alpha, beta, M, W, ldw, skip, s);
    case 16: return launch_update<T, BV, 16>(V, n, C, alpha, beta, M, W, ldw, skip, s);
  }
  return set_error(FE_ERR_INVALID, "update: bw = %d", bw);
}

int update_skip(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                const double* M, void* W, int bw, int ldw, fe_dtype dt, const int* skip,
                cudaStream_t s) {
  FE_ARG(V.nv >= 0 && V.nv <= kMaxBlocks, "update: nv = %d", V.nv);
  const int bv = V.nv > 0 ? V.bv : 1;
  if (dt == FE_F32) {
    float* w = static_cast<float*>(W);
    switch (bv) {
      case 1: return update_bv<float, 1>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 2: return update_bv<float, 2>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 4: return update_bv<float, 4>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 8: return update_bv<float, 8>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 16: return update_bv<float, 16>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
    }
  } else {
    double* w = static_cast<double*>(W);
    switch (bv) {
      case 1: return update_bv<double, 1>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 2: return update_bv<double, 2>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 4: return update_bv<double, 4>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 8: return update_bv<double, 8>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
      case 16: return update_bv<double, 16>(V, n, C, alpha, beta, M, w, bw, ldw, skip, s);
    }
  }
  return set_error(FE_ERR_INVALID, "update: bv = %d", bv);
}

int update(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
           const double* M, void* W, int bw, int ldw, fe_dtype dt, cudaStream_t s) {
  return update_skip(V, n, C, alpha, beta, M, W, bw, ldw, dt, nullptr, s);
}

// ---------------------------------------------------------------- combine (V Y)
// Out_o[r] = sum_j V_j[r] Y[j-block rows, o-block columns], thread per row.  Up to OB output
// blocks are accumulated in registers at once, so each V row is loaded once per group of OB
// output blocks (one group for the solver's restarts), two or four rows in flight.
template <typename T, int BV, int OB>
__global__ void __launch_bounds__(256) combine_kernel(const BlockSet V, const double* __restrict__ Y,
                                                      int ldy, const BlockSet Out, int64_t n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sY = reinterpret_cast<T*>(smem_raw);
  const int k = V.nv * BV, kout = Out.nv * BV;
  for (int e = threadIdx.x; e < k * kout; e += blockDim.x) sY[e] = (T)Y[(e / kout) * ldy + e % kout];
  __syncthreads();
  constexpr int UJ = BV >= 8 ? 2 : 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    for (int o0 = 0; o0 < Out.nv; o0 += OB) {
      T acc[OB][BV];
#pragma unroll
      for (int o = 0; o < OB; ++o)
#pragma unroll
        for (int q = 0; q < BV; ++q) acc[o][q] = T(0);
      for (int j0 = 0; j0 < V.nv; j0 += UJ) {
        T v[UJ][BV];
#pragma unroll
        for (int u = 0; u < UJ; ++u)
          if (j0 + u < V.nv) load_vrow<T, BV>(reinterpret_cast<const T*>(V.blk[j0 + u]), V.ld, r, v[u]);
#pragma unroll
        for (int u = 0; u < UJ; ++u) {
          if (j0 + u >= V.nv) break;
          const T* yj = sY + (size_t)((j0 + u) * BV) * kout + o0 * BV;
#pragma unroll
          for (int o = 0; o < OB; ++o) {
            if (o0 + o >= Out.nv) break;
#pragma unroll
            for (int p = 0; p < BV; ++p)
#pragma unroll
              for (int q = 0; q < BV; ++q) acc[o][q] = fma(v[u][p], yj[p * kout + o * BV + q], acc[o][q]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < OB; ++o) {
        if (o0 + o >= Out.nv) break;
        T* dst = const_cast<T*>(reinterpret_cast<const T*>(Out.blk[o0 + o]));
        if (Out.ld == BV) {
          st_row<T, BV>(dst + r * BV, acc[o]);
        } else {
#pragma unroll
          for (int q = 0; q < BV; ++q) dst[r * Out.ld + q] = acc[o][q];
        }
      }
    }
  }
}

template <typename T, int BV>
static int launch_combine(const BlockSet& V, int64_t n, const double* Y, int ldy,
                          const BlockSet& Out, cudaStream_t s) {
  constexpr int OB = BV <= 4 ? 8 : (BV == 8 ? 4 : 2);
  static KernelSetup ks;
  FE_TRY(kernel_configure(ks, reinterpret_cast<const void*>(combine_kernel<T, BV, OB>), 200 * 1024));
  int ctas = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
  ctas = std::max(ctas, 1);
  // the coefficients of at most `per` output blocks at a time in shared memory (large subspaces
  // take several launches, each reading V again)
  const size_t per_block = (size_t)V.nv * BV * BV * sizeof(T);
  const int per = (int)std::max<size_t>(1, std::min<size_t>(Out.nv, (size_t)(160 * 1024) / per_block));
  FE_ARG(per_block <= 200 * 1024, "combine: coefficient matrix too large");
  for (int o0 = 0; o0 < Out.nv; o0 += per) {
    BlockSet sub = Out;
    sub.nv = std::min(per, Out.nv - o0);
    for (int o = 0; o < sub.nv; ++o) sub.blk[o] = Out.blk[o0 + o];
    const size_t smem = per_block * sub.nv;
    combine_kernel<T, BV, OB><<<ctas, 256, smem, s>>>(V, Y + (size_t)o0 * BV, ldy, sub, n);
    count_launch();
    FE_CUDA(cudaGetLastError());
  }
  return FE_OK;
}

int combine(const BlockSet& V, int64_t n, const double* Y, int ldy, const BlockSet& Out,
            fe_dtype dt, cudaStream_t s, int engine) {
  FE_ARG(V.bv == Out.bv, "combine: block widths differ");
  FE_ARG(V.nv >= 1 && Out.nv >= 1, "combine: empty block set");
  FE_ARG(engine == FE_ENGINE_AUTO || engine == FE_ENGINE_FMA || engine == FE_ENGINE_TC,
         "combine: engine = %d", engine);
  if (engine != FE_ENGINE_FMA && dt == FE_F64) {
    if (tc_combine_supported(V, Out, dt)) return tc_combine(V, n, Y, ldy, Out, s);
    FE_ARG(engine == FE_ENGINE_AUTO,
           "combine: the tensor-core engine takes FP64 blocks with nv*bv <= 64 and nout*bv <= 32");
  }
  FE_ARG(engine != FE_ENGINE_TC, "combine: the tensor-core engine takes FP64 blocks only");
  if (dt == FE_F32) {
    switch (V.bv) {
      case 1: return launch_combine<float, 1>(V, n, Y, ldy, Out, s);
      case 2: return launch_combine<float, 2>(V, n, Y, ldy, Out, s);
      case 4: return launch_combine<float, 4>(V, n, Y, ldy, Out, s);
      case 8: return launch_combine<float, 8>(V, n, Y, ldy, Out, s);
      case 16: return launch_combine<float, 16>(V, n, Y, ldy, Out, s);
    }
  } else {
    switch (V.bv) {
      case 1: return launch_combine<double, 1>(V, n, Y, ldy, Out, s);
      case 2: return launch_combine<double, 2>(V, n, Y, ldy, Out, s);
      case 4: return launch_combine<double, 4>(V, n, Y, ldy, Out, s);
      case 8: return launch_combine<double, 8>(V, n, Y, ldy, Out, s);
      case 16: return launch_combine<double, 16>(V, n, Y, ldy, Out, s);
    }
  }
  return set_error(FE_ERR_INVALID, "combine: bv = %d", V.bv);
}

// ---------------------------------------------------------------- MvRandom
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a hash of (seed, stream, counter),
// Box-Muller (1958) for the normal deviate.
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sm64_u01(uint64_t s0, uint64_t i) {
  return (double)(sm64_mix(s0 + (i + 1) * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
}

template <typename T>
__global__ void random_normal_kernel(T* __restrict__ X, int64_t n, int b, int ld, uint64_t s0,
                                     uint64_t offset) {
  const int64_t total = n * b;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint64_t idx = offset + (uint64_t)i;
    const double u1 = sm64_u01(s0, 2 * idx);
    const double u2 = sm64_u01(s0, 2 * idx + 1);
    const double z = sqrt(-2.0 * log1p(-u1)) * cos(2.0 * 3.14159265358979323846 * u2);
    X[(i / b) * ld + (i % b)] = (T)z;
  }
}

static uint64_t host_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int random_normal(void* X, int64_t n, int b, int ld, fe_dtype dt, uint64_t seed, uint64_t stream,
                  uint64_t offset, cudaStream_t s) {
  const uint64_t s0 = host_mix(seed * 0x9E3779B97F4A7C15ull + stream * 0xD1B54A32D192ED03ull +
                               0x632BE59BD9B4E019ull);
  int ctas = (int)std::min<int64_t>(ceil_div(n * b, 256), 8 * num_sms());
  ctas = std::max(ctas, 1);
  if (dt == FE_F32)
    random_normal_kernel<float><<<ctas, 256, 0, s>>>(static_cast<float*>(X), n, b, ld, s0, offset);
  else
    random_normal_kernel<double><<<ctas, 256, 0, s>>>(static_cast<double*>(X), n, b, ld, s0, offset);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// ---------------------------------------------------------------- layout / type conversions
// dst[r*ldd + c] = src[r*lds + c], element types converted.
template <typename S, typename D>
__global__ void cast_rows_kernel(const S* __restrict__ src, int lds, D* __restrict__ dst, int ldd,
                                 int64_t n, int b) {
  const int64_t total = n * b;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    dst[(i / b) * ldd + i % b] = (D)src[(i / b) * lds + i % b];
}

int convert_block(const void* src, fe_dtype sdt, int lds, void* dst, fe_dtype ddt, int ldd,
                  int64_t n, int b, cudaStream_t s) {
  int ctas = (int)std::min<int64_t>(ceil_div(n * b, 256), 8 * num_sms());
  ctas = std::max(ctas, 1);
  if (sdt == FE_F64 && ddt == FE_F64)
    cast_rows_kernel<double, double><<<ctas, 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, n, b);
  else if (sdt == FE_F64 && ddt == FE_F32)
    cast_rows_kernel<double, float><<<ctas, 256, 0, s>>>((const double*)src, lds, (float*)dst, ldd, n, b);
  else if (sdt == FE_F32 && ddt == FE_F64)
    cast_rows_kernel<float, double><<<ctas, 256, 0, s>>>((const float*)src, lds, (double*)dst, ldd, n, b);
  else
    cast_rows_kernel<float, float><<<ctas, 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, n, b);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// out[c*n + r] = column c of the block set (ConvLayout, Table 1: row-major -> column-major).
template <typename T>
__global__ void to_colmajor_kernel(const BlockSet X, int64_t n, int ncols, double* __restrict__ out) {
  const int64_t total = n * ncols;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int c = (int)(i / n);
    const int64_t r = i % n;
    const T* blk = reinterpret_cast<const T*>(X.blk[c / X.bv]);
    out[i] = (double)blk[r * X.ld + c % X.bv];
  }
}

int to_colmajor_f64(const BlockSet& X, int64_t n, int ncols, fe_dtype dt, double* out,
                    cudaStream_t s) {
  int ctas = (int)std::min<int64_t>(ceil_div(n * ncols, 256), 8 * num_sms());
  ctas = std::max(ctas, 1);
  if (dt == FE_F32) to_colmajor_kernel<float><<<ctas, 256, 0, s>>>(X, n, ncols, out);
  else to_colmajor_kernel<double><<<ctas, 256, 0, s>>>(X, n, ncols, out);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

}  // namespace fe

namespace fe {

// ---------------------------------------------------------------- gram into given scratch
// Same kernels as gram(), but the per-CTA partials go to `scratch` (capacity doubles) supplied
// by the caller, and nothing is allocated here.  The grid shrinks so the partials fit.
template <typename T, int BV, int NQ>
static int launch_gram_scratch(const BlockSet& V, int64_t n, const T* W, int bw, int ldw,
                               double alpha, double* G, double* scratch, size_t capacity,
                               cudaStream_t s) {
  FE_ARG(scratch != nullptr, "gram: NULL scratch");
  return launch_gram_any<T, BV, NQ>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
}

template <typename T, int BV>
static int gram_scratch_bv(const BlockSet& V, int64_t n, const T* W, int bw, int ldw,
                           double alpha, double* G, double* scratch, size_t capacity,
                           cudaStream_t s) {
  constexpr int QMAX = 32 / BV >= 16 ? 16 : 32 / BV;
  const int nq = std::min(bw, QMAX);
  switch (nq) {
    case 1: return launch_gram_scratch<T, BV, 1>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
    case 2: return launch_gram_scratch<T, BV, (QMAX >= 2 ? 2 : 1)>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
    case 4: return launch_gram_scratch<T, BV, (QMAX >= 4 ? 4 : 1)>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
    case 8: return launch_gram_scratch<T, BV, (QMAX >= 8 ? 8 : 1)>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
    case 16: return launch_gram_scratch<T, BV, (QMAX >= 16 ? 16 : 1)>(V, n, W, bw, ldw, alpha, G, scratch, capacity, s);
  }
  return set_error(FE_ERR_INVALID, "gram: bad bw %d", bw);
}

int gram_into_scratch(const BlockSet& V, int64_t n, const void* W, int bw, int ldw, fe_dtype dt,
                      double alpha, double* G, double* scratch, size_t capacity, cudaStream_t s) {
  FE_ARG(V.nv >= 1 && V.nv <= kMaxBlocks, "gram: nv = %d out of range", V.nv);
  FE_ARG(is_pow2_le16(bw), "gram: bw = %d", bw);
  if (dt == FE_F32) {
    const float* w = static_cast<const float*>(W);
    switch (V.bv) {
      case 1: return gram_scratch_bv<float, 1>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 2: return gram_scratch_bv<float, 2>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 4: return gram_scratch_bv<float, 4>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 8: return gram_scratch_bv<float, 8>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 16: return gram_scratch_bv<float, 16>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
    }
  } else {
    const double* w = static_cast<const double*>(W);
    switch (V.bv) {
      case 1: return gram_scratch_bv<double, 1>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 2: return gram_scratch_bv<double, 2>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 4: return gram_scratch_bv<double, 4>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 8: return gram_scratch_bv<double, 8>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
      case 16: return gram_scratch_bv<double, 16>(V, n, w, bw, ldw, alpha, G, scratch, capacity, s);
    }
  }
  return set_error(FE_ERR_INVALID, "gram: bv = %d not in {1,2,4,8,16}", V.bv);
}

}  // namespace fe

namespace fe {

// ---------------------------------------------------------------- fused update + Gram
// One sweep over the rows: W[r] = beta (W[r] M) + alpha sum_j V_j[r] C_j (thread per row, as
// update_kernel), then the Gram partials of [V_0 .. V_{nv-1}, W_new]^T W_new (only of W_new^T
// W_new when gram_v == 0), accumulated per CTA like gram_kernel.  Phase A leaves the range's
// new W rows in shared memory (two buffers, so one barrier per range suffices); phase B re-reads
// the range's V rows, which phase A has just pulled into L1, so V comes from DRAM once for both
// operations.  Gram tiles are the V blocks then W_new; TPW > 0: warp w owns tiles w + nwarps t
// for the whole launch and reduces once at the end (the block has one warp per tile, up to 16,
// and a range is one row per thread); TPW == 0: 8 warps, tiles reduced per range.
//
// vc32 (FP64 only): when *vc32 != 0 the sum alpha sum_j V_j[r] C_j is formed in FP32 arithmetic
// (V converted by f64_to_f32_trunc, FP32 coefficients, FP32 accumulation) and added to the FP64
// W[r] M.  The caller sets the flag only when the coefficients are tiny corrections (the second
// Gram-Schmidt pass), so that the FP32 rounding stays far below FP64 rounding of W.
template <typename T, int BV, int BW, int TPW>
__global__ void __launch_bounds__(TPW > 0 ? 512 : 256) update_gram_kernel(const BlockSet V, const double* __restrict__ C,
                                                          double alpha, double beta,
                                                          const double* __restrict__ M,
                                                          T* __restrict__ W, int64_t n, int gram_v,
                                                          const int* __restrict__ skip,
                                                          const int* __restrict__ vc32,
                                                          double* __restrict__ partial) {
  if (skip && *skip) return;
  const bool use32 = sizeof(T) == 8 && vc32 != nullptr && *vc32 != 0;
  const int R = blockDim.x;
  const int kWarps = blockDim.x >> 5;
  constexpr int NR = BV > BW ? BV : BW;
  constexpr int NT = TPW > 0 ? TPW : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = V.nv * BV;
  T* sC = reinterpret_cast<T*>(smem_raw);
  T* sM = sC + (size_t)k * BW;
  T* sW = sM + BW * BW;  // two buffers of R x BW
  double* sP = reinterpret_cast<double*>(smem_raw + ((((size_t)k * BW + BW * BW + 2 * (size_t)R * BW) * sizeof(T) + 15) & ~(size_t)15));
  const int gblocks = gram_v ? V.nv + 1 : 1;  // Gram row blocks: the V blocks (if any), then W
  const int nout = (gram_v ? k : 0) * BW + BW * BW;
  float* sC32 = reinterpret_cast<float*>(sP + nout);  // FP32 coefficients (vc32 launches)
  for (int e = threadIdx.x; e < k * BW; e += blockDim.x) sC[e] = (T)(alpha * C[e]);
  if (vc32)
    for (int e = threadIdx.x; e < k * BW; e += blockDim.x) sC32[e] = (float)(alpha * C[e]);
  if (M)
    for (int e = threadIdx.x; e < BW * BW; e += blockDim.x) sM[e] = (T)(beta * M[e]);
  for (int e = threadIdx.x; e < nout; e += blockDim.x) sP[e] = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T acc[NT][NR][BW];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int p = 0; p < NR; ++p)
#pragma unroll
      for (int q = 0; q < BW; ++q) acc[t][p][q] = T(0);
  __syncthreads();  // coefficients loaded
  int buf = 0;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < n; r0 += (int64_t)gridDim.x * R, buf ^= 1) {
    const int rows = (int)min((int64_t)R, n - r0);
    T* sWb = sW + buf * R * BW;
    // phase A: update (thread per row), V rows four blocks at a time
    if ((int)threadIdx.x < rows) {
      const int64_t r = r0 + threadIdx.x;
      T a[BW];
      if (beta == 0.0) {
#pragma unroll
        for (int q = 0; q < BW; ++q) a[q] = T(0);
      } else {
        T w[BW];
        ld_row_rw<T, BW>(W + r * BW, w);
        if (M) {
#pragma unroll
          for (int q = 0; q < BW; ++q) {
            T x = T(0);
#pragma unroll
            for (int p = 0; p < BW; ++p) x = fma(w[p], sM[p * BW + q], x);
            a[q] = x;
          }
        } else {
#pragma unroll
          for (int q = 0; q < BW; ++q) a[q] = (T)beta * w[q];
        }
      }
      constexpr int UJ = BV >= 8 ? 2 : 4;
      if (use32) {
        float a32[BW];
#pragma unroll
        for (int q = 0; q < BW; ++q) a32[q] = 0.f;
        for (int j0 = 0; j0 < V.nv; j0 += UJ) {
          T v[UJ][BV];
#pragma unroll
          for (int u = 0; u < UJ; ++u)
            if (j0 + u < V.nv) load_vrow<T, BV>(reinterpret_cast<const T*>(V.blk[j0 + u]), V.ld, r, v[u]);
#pragma unroll
          for (int u = 0; u < UJ; ++u) {
            if (j0 + u < V.nv) {
              const float* c = sC32 + (j0 + u) * BV * BW;
#pragma unroll
              for (int p = 0; p < BV; ++p) {
                const float vp = f64_to_f32_trunc((double)v[u][p]);
#pragma unroll
                for (int q = 0; q < BW; ++q) a32[q] = fmaf(vp, c[p * BW + q], a32[q]);
              }
            }
          }
        }
#pragma unroll
        for (int q = 0; q < BW; ++q) a[q] += (T)f32_to_f64_flush(a32[q]);
      } else {
        for (int j0 = 0; j0 < V.nv; j0 += UJ) {
          T v[UJ][BV];
#pragma unroll
          for (int u = 0; u < UJ; ++u)
            if (j0 + u < V.nv) load_vrow<T, BV>(reinterpret_cast<const T*>(V.blk[j0 + u]), V.ld, r, v[u]);
#pragma unroll
          for (int u = 0; u < UJ; ++u) {
            if (j0 + u < V.nv) {
              const T* c = sC + (j0 + u) * BV * BW;
#pragma unroll
              for (int p = 0; p < BV; ++p)
#pragma unroll
                for (int q = 0; q < BW; ++q) a[q] = fma(v[u][p], c[p * BW + q], a[q]);
            }
          }
        }
      }
      st_row<T, BW>(W + r * BW, a);
#pragma unroll
      for (int q = 0; q < BW; ++q) sWb[threadIdx.x * BW + q] = a[q];
    }
    __syncthreads();
    // phase B: Gram tiles (warp per tile, lane = row)
    auto sweep = [&](int tile, T (&ac)[NR][BW]) {
      const bool isW = tile == gblocks - 1;
      if (isW) {
        for (int r = lane; r < rows; r += 32) {
          T wq[BW];
#pragma unroll
          for (int q = 0; q < BW; ++q) wq[q] = sWb[r * BW + q];
#pragma unroll
          for (int p = 0; p < BW; ++p)
#pragma unroll
            for (int q = 0; q < BW; ++q) ac[p][q] = fma(wq[p], wq[q], ac[p][q]);
        }
      } else {
        const T* vb = reinterpret_cast<const T*>(V.blk[tile]);
        for (int r = lane; r < rows; r += 32) {
          T v[BV];
          load_vrow<T, BV>(vb, V.ld, r0 + r, v);
          T wq[BW];
#pragma unroll
          for (int q = 0; q < BW; ++q) wq[q] = sWb[r * BW + q];
#pragma unroll
          for (int p = 0; p < BV; ++p)
#pragma unroll
            for (int q = 0; q < BW; ++q) ac[p][q] = fma(v[p], wq[q], ac[p][q]);
        }
      }
    };
    auto flush = [&](int tile, T (&ac)[NR][BW]) {
      const bool isW = tile == gblocks - 1;
      const int np = isW ? BW : BV;
      const int rowoff = isW ? (gram_v ? k : 0) : tile * BV;
#pragma unroll
      for (int p = 0; p < NR; ++p) {
        if (p >= np) break;
#pragma unroll
        for (int q = 0; q < BW; ++q) {
          double x = (double)ac[p][q];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFullMask, x, off);
          if (lane == 0) sP[(rowoff + p) * BW + q] += x;
          ac[p][q] = T(0);
        }
      }
    };
    if (TPW > 0) {
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (warp + kWarps * t < gblocks) sweep(warp + kWarps * t, acc[t]);
    } else {
      for (int tile = warp; tile < gblocks; tile += kWarps) {
        sweep(tile, acc[0]);
        flush(tile, acc[0]);
      }
    }
    if (r0 + (int64_t)gridDim.x * R >= n && TPW > 0) {
      // last range of this CTA: reduce the persistent accumulators
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (warp + kWarps * t < gblocks) flush(warp + kWarps * t, acc[t]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nout; e += blockDim.x) partial[(int64_t)blockIdx.x * nout + e] = sP[e];
}

template <typename T, int BV, int BW, int TPW>
static int launch_update_gram_tpw(const BlockSet& V, int64_t n, const double* C, double alpha,
                                  double beta, const double* M, T* W, int gram_v, const int* skip,
                                  const int* vc32, double* G, int threads, cudaStream_t s) {
  const int R = threads;
  const int k = V.nv * BV;
  const int nout = (gram_v ? k : 0) * BW + BW * BW;
  const size_t smem = ((((size_t)k * BW + BW * BW + 2 * (size_t)R * BW) * sizeof(T) + 15) & ~(size_t)15) +
                      (size_t)nout * sizeof(double) + (vc32 ? (size_t)k * BW * sizeof(float) : 0);
  FE_ARG(smem <= 200 * 1024, "update_gram: coefficient matrix too large");
  static KernelSetup ks;
  const void* fn = reinterpret_cast<const void*>(update_gram_kernel<T, BV, BW, TPW>);
  FE_TRY(kernel_configure(ks, fn, 200 * 1024));
  const int wq = threads / 32;  // launch shape: warps per block
  FE_ARG(threads % 32 == 0 && wq >= 8 && wq <= 16, "update_gram: %d threads", threads);
  int per_sm = 0;
  FE_TRY(kernel_occupancy(ks, fn, threads, smem, wq, &per_sm));
  int nctas = (int)std::min<int64_t>(ceil_div(n, R), (int64_t)per_sm * num_sms());
  nctas = std::max(nctas, 1);
  double* part = small_scratch(0, (size_t)nctas * nout);
  if (!part) return FE_ERR_OOM;
  update_gram_kernel<T, BV, BW, TPW><<<nctas, threads, smem, s>>>(V, C, alpha, beta, M, W, n, gram_v, skip, vc32, part);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return launch_gram_reduce(part, nctas, nout, 1.0, G, s);
}

// One warp per Gram tile with persistent accumulators (up to 16 tiles, 32 32-bit registers
// per tile); otherwise 8 warps reducing per range.
template <typename T, int BV, int BW>
static int launch_update_gram(const BlockSet& V, int64_t n, const double* C, double alpha,
                              double beta, const double* M, T* W, int gram_v, const int* skip,
                              const int* vc32, double* G, cudaStream_t s) {
  constexpr int NR = BV > BW ? BV : BW;
  constexpr int kRegsPerTile = NR * BW * (int)(sizeof(T) / 4);
  const int gblocks = gram_v ? V.nv + 1 : 1;
  if (gblocks <= 16 && kRegsPerTile <= 32)
    return launch_update_gram_tpw<T, BV, BW, (kRegsPerTile <= 32 ? 1 : 0)>(
        V, n, C, alpha, beta, M, W, gram_v, skip, vc32, G, 32 * std::max(8, gblocks), s);
  return launch_update_gram_tpw<T, BV, BW, 0>(V, n, C, alpha, beta, M, W, gram_v, skip, vc32, G, 256, s);
}

// The second Gram-Schmidt pass's closing sweep for blocks of width B <= 4, with M upper
// triangular (M = R1^{-1} of the CholeskyQR pass): W = beta W M + alpha V C and S = W^T W (after
// the update).  Thread per row: the triangle of M (B (B + 1) / 2 FMAs instead of B^2); for FP64
// blocks the correction V C in FP32 arithmetic when *vc32 (its entries are tiny; V read through
// an integer truncation to FP32, added to the FP64 W M in FP64), otherwise in T; the upper
// triangle of S in per-thread accumulators (T) over the rows the thread visits (a grid-stride
// loop), reduced over the CTA in FP64 and written as the CTA's full B x B partial.  *skip:
// nothing done.
template <typename T, int B>
__global__ void __launch_bounds__(256) update_tri_gram_kernel(const BlockSet V, const double* __restrict__ C,
                                                             double alpha, double beta,
                                                             const double* __restrict__ M,
                                                             T* __restrict__ W, int64_t n,
                                                             const int* __restrict__ skip,
                                                             const int* __restrict__ vc32,
                                                             double* __restrict__ partial) {
  if (skip && *skip) return;
  constexpr int NS = B * (B + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = V.nv * B;
  double* sR = reinterpret_cast<double*>(smem_raw);            // [warps][NS] reduction
  T* sC = reinterpret_cast<T*>(sR + (blockDim.x / 32) * NS);   // k x B
  T* sM = sC + (size_t)k * B;                                  // B x B
  float* sC32 = reinterpret_cast<float*>(sM + B * B);
  const bool use32 = sizeof(T) == 8 && vc32 != nullptr && *vc32 != 0;
  for (int e = threadIdx.x; e < k * B; e += blockDim.x) {
    sC[e] = (T)(alpha * C[e]);
    sC32[e] = (float)(alpha * C[e]);
  }
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) sM[e] = (T)(beta * M[e]);
  __syncthreads();
  T acc[NS];
#pragma unroll
  for (int e = 0; e < NS; ++e) acc[e] = T(0);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    T w[B], a[B];
    ld_row_rw<T, B>(W + r * B, w);
#pragma unroll
    for (int q = 0; q < B; ++q) {
      T x = T(0);
#pragma unroll
      for (int p = 0; p <= q; ++p) x = fma(w[p], sM[p * B + q], x);
      a[q] = x;
    }
    if (use32) {
      float a32[B];
#pragma unroll
      for (int q = 0; q < B; ++q) a32[q] = 0.f;
      for (int j = 0; j < V.nv; ++j) {
        T v[B];
        ld_row<T, B>(reinterpret_cast<const T*>(V.blk[j]) + r * B, v);
#pragma unroll
        for (int p = 0; p < B; ++p) {
          const float vp = to_arith<float>(v[p]);
#pragma unroll
          for (int q = 0; q < B; ++q) a32[q] = fmaf(vp, sC32[(j * B + p) * B + q], a32[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < B; ++q) a[q] += (T)f32_to_f64_flush(a32[q]);
    } else {
      for (int j = 0; j < V.nv; ++j) {
        T v[B];
        ld_row<T, B>(reinterpret_cast<const T*>(V.blk[j]) + r * B, v);
#pragma unroll
        for (int p = 0; p < B; ++p)
#pragma unroll
          for (int q = 0; q < B; ++q) a[q] = fma(v[p], sC[(j * B + p) * B + q], a[q]);
      }
    }
    st_row<T, B>(W + r * B, a);
    int e = 0;
#pragma unroll
    for (int p = 0; p < B; ++p)
#pragma unroll
      for (int q = p; q < B; ++q, ++e) acc[e] = fma(a[p], a[q], acc[e]);
  }
  // CTA reduction of the triangle in FP64 (warp shuffles, then the warps' sums in a fixed order)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int e = 0; e < NS; ++e) {
    double x = (double)acc[e];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) sR[warp * NS + e] = x;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double x = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x / 32); ++w2) x += sR[w2 * NS + threadIdx.x];
    int p = 0, e = threadIdx.x;
    while (e >= B - p) { e -= B - p; ++p; }
    const int q = p + e;
    partial[(int64_t)blockIdx.x * B * B + p * B + q] = x;
    partial[(int64_t)blockIdx.x * B * B + q * B + p] = x;
  }
}

template <typename T>
static int launch_update_tri_gram(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                                  const double* M, T* W, int b, const int* skip, const int* vc32, double* S,
                                  cudaStream_t s) {
  const int k = V.nv * b;
  const int threads = 256;
  const int NS = b * (b + 1) / 2;
  const size_t smem = (size_t)(threads / 32) * NS * sizeof(double) + ((size_t)k * b + b * b) * sizeof(T) +
                      (size_t)k * b * sizeof(float);
  const void* fn = b == 1 ? reinterpret_cast<const void*>(update_tri_gram_kernel<T, 1>)
                 : b == 2 ? reinterpret_cast<const void*>(update_tri_gram_kernel<T, 2>)
                          : reinterpret_cast<const void*>(update_tri_gram_kernel<T, 4>);
  static KernelSetup ks[3];
  const int bi = b == 1 ? 0 : b == 2 ? 1 : 2;
  FE_TRY(kernel_configure(ks[bi], fn, 96 * 1024));
  int per_sm = 0;
  FE_TRY(kernel_occupancy(ks[bi], fn, threads, smem, 0, &per_sm));
  const int nctas = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)per_sm * num_sms()));
  double* part = small_scratch(0, (size_t)nctas * b * b);
  if (!part) return FE_ERR_OOM;
  switch (b) {
    case 1: update_tri_gram_kernel<T, 1><<<nctas, threads, smem, s>>>(V, C, alpha, beta, M, W, n, skip, vc32, part); break;
    case 2: update_tri_gram_kernel<T, 2><<<nctas, threads, smem, s>>>(V, C, alpha, beta, M, W, n, skip, vc32, part); break;
    default: update_tri_gram_kernel<T, 4><<<nctas, threads, smem, s>>>(V, C, alpha, beta, M, W, n, skip, vc32, part); break;
  }
  count_launch();
  FE_CUDA(cudaGetLastError());
  return launch_gram_reduce(part, nctas, b * b, 1.0, S, s);
}

// W = beta W M + alpha V C, S = W^T W for n x b blocks of dt, b in {1, 2, 4}, M upper triangular
// (see update_tri_gram_kernel); S: DEVICE b x b.
int update_tri_gram(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                    const double* M, void* W, int b, fe_dtype dt, const int* skip, const int* vc32, double* S,
                    cudaStream_t s) {
  FE_ARG(b == 1 || b == 2 || b == 4, "update_tri_gram: b = %d", b);
  FE_ARG(V.nv == 0 || (V.bv == b && V.ld == b), "update_tri_gram: blocks must be n x b");
  if (dt == FE_F64)
    return launch_update_tri_gram<double>(V, n, C, alpha, beta, M, static_cast<double*>(W), b, skip, vc32, S, s);
  return launch_update_tri_gram<float>(V, n, C, alpha, beta, M, static_cast<float*>(W), b, skip, nullptr, S, s);
}

// W = beta W M + alpha V C; G = [V; W]^T W (gram_v) or W^T W, rows (j*b + p) then W's b rows.
// V blocks and W must all be n x b with ld b (the solver's subspace blocks).
int update_gram(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                const double* M, void* W, int b, fe_dtype dt, int gram_v, const int* skip,
                double* G, cudaStream_t s, const int* vc32) {
  FE_ARG(V.nv >= 0 && V.nv <= kMaxBlocks, "update_gram: nv = %d", V.nv);
  FE_ARG(V.nv == 0 || (V.bv == b && V.ld == b), "update_gram: blocks must be n x b");
  if (dt != FE_F64) vc32 = nullptr;
#define UG(T, B) return launch_update_gram<T, B, B>(V, n, C, alpha, beta, M, static_cast<T*>(W), gram_v, skip, vc32, G, s)
  if (dt == FE_F32) {
    switch (b) { case 1: UG(float, 1); case 2: UG(float, 2); case 4: UG(float, 4); case 8: UG(float, 8); }
  } else {
    switch (b) { case 1: UG(double, 1); case 2: UG(double, 2); case 4: UG(double, 4); case 8: UG(double, 8); }
  }
#undef UG
  return set_error(FE_ERR_INVALID, "update_gram: b = %d not in {1, 2, 4, 8}", b);
}

}  // namespace fe
