// Dense tall-and-skinny block operations of Table 1 on row-major n x b blocks.
//
//   gram     MvTransMv ("op3"): G = alpha V^T W.  Two phases as in Section 3.4.2 (each CTA
//            reduces its row ranges to a small partial matrix, then one pass adds the partials
//            in CTA order -- deterministic, no atomics).  Inside a CTA a range of W rows is
//            staged in shared memory once; each warp owns one (block j, column group) output
//            tile and sweeps the range with lane = row, so every V element is read once,
//            coalesced.
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
static thread_local ScratchPool* t_pool = nullptr;
static thread_local int t_pool_dev = -1;

static ScratchPool& pool() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (!t_pool || t_pool_dev != dev) {
    t_pool = new ScratchPool();  // per thread and device; lives until exit
    t_pool_dev = dev;
  }
  return *t_pool;
}

double* small_scratch(int slot, size_t count) {
  if (slot < 0 || slot >= kScratchSlots) {
    set_error(FE_ERR_INVALID, "internal: scratch slot %d out of range", slot);
    return nullptr;
  }
  DevBuf& b = pool().bufs[slot];
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
template <typename T, int BV, int NQ>
__global__ void __launch_bounds__(256) gram_kernel(const BlockSet V, const T* __restrict__ W,
                                                   int ldw, int bw, int64_t n, int R,
                                                   double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);
  double* sP = reinterpret_cast<double*>(smem_raw + (((size_t)R * bw * sizeof(T) + 15) & ~(size_t)15));
  const int nout = V.nv * BV * bw;
  for (int e = threadIdx.x; e < nout; e += blockDim.x) sP[e] = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int qtiles = bw / NQ;
  const int ntiles = V.nv * qtiles;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < n; r0 += (int64_t)gridDim.x * R) {
    const int rows = (int)min((int64_t)R, n - r0);
    __syncthreads();
    const int tot = rows * bw;
    if (ldw == bw) {
      const T* src = W + r0 * bw;
      for (int e = threadIdx.x; e < tot; e += blockDim.x) sW[e] = src[e];
    } else {
      for (int e = threadIdx.x; e < tot; e += blockDim.x) sW[e] = W[(r0 + e / bw) * ldw + e % bw];
    }
    __syncthreads();
    for (int tile = warp; tile < ntiles; tile += nwarps) {
      const int j = tile / qtiles, q0 = (tile % qtiles) * NQ;
      const T* __restrict__ vb = reinterpret_cast<const T*>(V.blk[j]);
      T acc[BV][NQ];
#pragma unroll
      for (int p = 0; p < BV; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[p][q] = T(0);
      for (int r = lane; r < rows; r += 32) {
        T v[BV];
        load_vrow<T, BV>(vb, V.ld, r0 + r, v);
        const T* w = sW + r * bw + q0;
        T wq[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) wq[q] = w[q];
#pragma unroll
        for (int p = 0; p < BV; ++p)
#pragma unroll
          for (int q = 0; q < NQ; ++q) acc[p][q] = fma(v[p], wq[q], acc[p][q]);
      }
#pragma unroll
      for (int p = 0; p < BV; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          double a = (double)acc[p][q];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(kFullMask, a, off);
          if (lane == 0) sP[(j * BV + p) * bw + q0 + q] += a;
        }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nout; e += blockDim.x) partial[(int64_t)blockIdx.x * nout + e] = sP[e];
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nctas, int nout,
                                   double alpha, double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nout) return;
  double s = 0.0;
  for (int c = 0; c < nctas; ++c) s += partial[(int64_t)c * nout + e];
  G[e] = alpha * s;
}

template <typename T, int BV, int NQ>
static int launch_gram(const BlockSet& V, int64_t n, const T* W, int bw, int ldw, double alpha,
                       double* G, cudaStream_t s) {
  const int nout = V.nv * BV * bw;
  int R = (int)(32768 / ((size_t)bw * sizeof(T)));
  R = std::max(32, R - R % 32);
  const size_t smem = (((size_t)R * bw * sizeof(T) + 15) & ~(size_t)15) + (size_t)nout * sizeof(double);
  FE_ARG(smem <= 200 * 1024, "gram: output too large (%d entries)", nout);
  static bool configured = false;  // per instantiation
  if (!configured) {
    FE_CUDA(cudaFuncSetAttribute(gram_kernel<T, BV, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  int nctas = (int)std::min<int64_t>(ceil_div(n, R), 2 * num_sms());
  nctas = std::max(nctas, 1);
  double* part = small_scratch(0, (size_t)nctas * nout);
  if (!part) return FE_ERR_OOM;
  gram_kernel<T, BV, NQ><<<nctas, 256, smem, s>>>(V, W, ldw, bw, n, R, part);
  count_launch();
  FE_CUDA(cudaGetLastError());
  gram_reduce_kernel<<<(unsigned)ceil_div(nout, 128), 128, 0, s>>>(part, nctas, nout, alpha, G);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
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
         double* G, cudaStream_t s) {
  FE_ARG(V.nv >= 1 && V.nv <= kMaxBlocks, "gram: nv = %d out of range", V.nv);
  FE_ARG(is_pow2_le16(bw), "gram: bw = %d", bw);
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
  static bool configured = false;
  if (!configured) {
    FE_CUDA(cudaFuncSetAttribute(update_kernel<T, BV, BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
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
template <typename T, int BV>
__global__ void __launch_bounds__(256) combine_kernel(const BlockSet V, const double* __restrict__ Y,
                                                      int ldy, const BlockSet Out, int64_t n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sY = reinterpret_cast<T*>(smem_raw);
  const int k = V.nv * BV, kout = Out.nv * BV;
  for (int e = threadIdx.x; e < k * kout; e += blockDim.x) sY[e] = (T)Y[(e / kout) * ldy + e % kout];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    for (int o = 0; o < Out.nv; ++o) {
      T acc[BV];
#pragma unroll
      for (int q = 0; q < BV; ++q) acc[q] = T(0);
      for (int j = 0; j < V.nv; ++j) {
        T v[BV];
        load_vrow<T, BV>(reinterpret_cast<const T*>(V.blk[j]), V.ld, r, v);
        const T* y = sY + (size_t)(j * BV) * kout + o * BV;
#pragma unroll
        for (int p = 0; p < BV; ++p)
#pragma unroll
          for (int q = 0; q < BV; ++q) acc[q] = fma(v[p], y[p * kout + q], acc[q]);
      }
      T* dst = const_cast<T*>(reinterpret_cast<const T*>(Out.blk[o]));
      if (Out.ld == BV) {
        st_row<T, BV>(dst + r * BV, acc);
      } else {
#pragma unroll
        for (int q = 0; q < BV; ++q) dst[r * Out.ld + q] = acc[q];
      }
    }
  }
}

template <typename T, int BV>
static int launch_combine(const BlockSet& V, int64_t n, const double* Y, int ldy,
                          const BlockSet& Out, cudaStream_t s) {
  const size_t smem = (size_t)V.nv * BV * Out.nv * BV * sizeof(T);
  FE_ARG(smem <= 200 * 1024, "combine: coefficient matrix too large");
  static bool configured = false;
  if (!configured) {
    FE_CUDA(cudaFuncSetAttribute(combine_kernel<T, BV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  int ctas = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
  ctas = std::max(ctas, 1);
  combine_kernel<T, BV><<<ctas, 256, smem, s>>>(V, Y, ldy, Out, n);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int combine(const BlockSet& V, int64_t n, const double* Y, int ldy, const BlockSet& Out,
            fe_dtype dt, cudaStream_t s) {
  FE_ARG(V.bv == Out.bv, "combine: block widths differ");
  FE_ARG(V.nv >= 1 && Out.nv >= 1, "combine: empty block set");
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
  const int nout = V.nv * BV * bw;
  int R = (int)(32768 / ((size_t)bw * sizeof(T)));
  R = std::max(32, R - R % 32);
  const size_t smem = (((size_t)R * bw * sizeof(T) + 15) & ~(size_t)15) + (size_t)nout * sizeof(double);
  FE_ARG(smem <= 200 * 1024, "gram: output too large (%d entries)", nout);
  static bool configured = false;
  if (!configured) {
    FE_CUDA(cudaFuncSetAttribute(gram_kernel<T, BV, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  int64_t nctas = std::min<int64_t>(ceil_div(n, R), 2 * num_sms());
  nctas = std::min<int64_t>(nctas, (int64_t)(capacity / (size_t)nout));
  FE_ARG(nctas >= 1, "gram: scratch of %zu doubles cannot hold %d outputs", capacity, nout);
  gram_kernel<T, BV, NQ><<<(unsigned)nctas, 256, smem, s>>>(V, W, ldw, bw, n, R, scratch);
  count_launch();
  FE_CUDA(cudaGetLastError());
  gram_reduce_kernel<<<(unsigned)ceil_div(nout, 128), 128, 0, s>>>(scratch, (int)nctas, nout, alpha, G);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
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
// W_new when gram_v == 0), accumulated per CTA like gram_kernel.  Phase A leaves the tile's new
// W rows in shared memory; phase B re-reads the tile's V rows, which phase A has just pulled
// into L1, so V comes from DRAM once for both operations.
template <typename T, int BV, int BW>
__global__ void __launch_bounds__(256) update_gram_kernel(const BlockSet V, const double* __restrict__ C,
                                                          double alpha, double beta,
                                                          const double* __restrict__ M,
                                                          T* __restrict__ W, int64_t n, int gram_v,
                                                          const int* __restrict__ skip,
                                                          double* __restrict__ partial) {
  if (skip && *skip) return;
  constexpr int R = 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = V.nv * BV;
  T* sC = reinterpret_cast<T*>(smem_raw);
  T* sM = sC + (size_t)k * BW;
  T* sW = sM + BW * BW;
  double* sP = reinterpret_cast<double*>(smem_raw + ((((size_t)k * BW + BW * BW + (size_t)R * BW) * sizeof(T) + 15) & ~(size_t)15));
  const int gblocks = gram_v ? V.nv + 1 : 1;  // Gram row blocks: the V blocks (if any), then W
  const int nout = (gram_v ? k : 0) * BW + BW * BW;
  for (int e = threadIdx.x; e < k * BW; e += blockDim.x) sC[e] = (T)(alpha * C[e]);
  if (M)
    for (int e = threadIdx.x; e < BW * BW; e += blockDim.x) sM[e] = (T)(beta * M[e]);
  for (int e = threadIdx.x; e < nout; e += blockDim.x) sP[e] = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < n; r0 += (int64_t)gridDim.x * R) {
    __syncthreads();  // coefficients loaded / previous tile's sW consumed
    const int rows = (int)min((int64_t)R, n - r0);
    // phase A: update (thread per row)
    if ((int)threadIdx.x < rows) {
      const int64_t r = r0 + threadIdx.x;
      T acc[BW];
      if (beta == 0.0) {
#pragma unroll
        for (int q = 0; q < BW; ++q) acc[q] = T(0);
      } else {
        T w[BW];
        ld_row_rw<T, BW>(W + r * BW, w);
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
      st_row<T, BW>(W + r * BW, acc);
#pragma unroll
      for (int q = 0; q < BW; ++q) sW[threadIdx.x * BW + q] = acc[q];
    }
    __syncthreads();
    // phase B: Gram tiles (warp per row block, lane = row)
    for (int tile = warp; tile < gblocks; tile += nwarps) {
      const bool isW = tile == gblocks - 1;
      const int j = tile;
      constexpr int NR = BV > BW ? BV : BW;
      T acc[NR][BW];
#pragma unroll
      for (int p = 0; p < NR; ++p)
#pragma unroll
        for (int q = 0; q < BW; ++q) acc[p][q] = T(0);
      for (int r = lane; r < rows; r += 32) {
        T wq[BW];
#pragma unroll
        for (int q = 0; q < BW; ++q) wq[q] = sW[r * BW + q];
        if (isW) {
#pragma unroll
          for (int p = 0; p < BW; ++p)
#pragma unroll
            for (int q = 0; q < BW; ++q) acc[p][q] = fma(wq[p], wq[q], acc[p][q]);
        } else {
          T v[BV];
          load_vrow<T, BV>(reinterpret_cast<const T*>(V.blk[j]), V.ld, r0 + r, v);
#pragma unroll
          for (int p = 0; p < BV; ++p)
#pragma unroll
            for (int q = 0; q < BW; ++q) acc[p][q] = fma(v[p], wq[q], acc[p][q]);
        }
      }
      const int np = isW ? BW : BV;
      const int rowoff = isW ? (gram_v ? k : 0) : j * BV;
#pragma unroll
      for (int p = 0; p < NR; ++p) {
        if (p >= np) break;
#pragma unroll
        for (int q = 0; q < BW; ++q) {
          double a = (double)acc[p][q];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(kFullMask, a, off);
          if (lane == 0) sP[(rowoff + p) * BW + q] += a;
        }
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nout; e += blockDim.x) partial[(int64_t)blockIdx.x * nout + e] = sP[e];
}

template <typename T, int BV, int BW>
static int launch_update_gram(const BlockSet& V, int64_t n, const double* C, double alpha,
                              double beta, const double* M, T* W, int gram_v, const int* skip,
                              double* G, cudaStream_t s) {
  constexpr int R = 256;
  const int k = V.nv * BV;
  const int nout = (gram_v ? k : 0) * BW + BW * BW;
  const size_t smem = ((((size_t)k * BW + BW * BW + (size_t)R * BW) * sizeof(T) + 15) & ~(size_t)15) +
                      (size_t)nout * sizeof(double);
  FE_ARG(smem <= 200 * 1024, "update_gram: coefficient matrix too large");
  static bool configured = false;
  if (!configured) {
    FE_CUDA(cudaFuncSetAttribute(update_gram_kernel<T, BV, BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  int nctas = (int)std::min<int64_t>(ceil_div(n, R), 2 * num_sms());
  nctas = std::max(nctas, 1);
  double* part = small_scratch(0, (size_t)nctas * nout);
  if (!part) return FE_ERR_OOM;
  update_gram_kernel<T, BV, BW><<<nctas, 256, smem, s>>>(V, C, alpha, beta, M, W, n, gram_v, skip, part);
  count_launch();
  FE_CUDA(cudaGetLastError());
  gram_reduce_kernel<<<(unsigned)ceil_div(nout, 128), 128, 0, s>>>(part, nctas, nout, 1.0, G);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// W = beta W M + alpha V C; G = [V; W]^T W (gram_v) or W^T W, rows (j*b + p) then W's b rows.
// V blocks and W must all be n x b with ld b (the solver's subspace blocks).
int update_gram(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                const double* M, void* W, int b, fe_dtype dt, int gram_v, const int* skip,
                double* G, cudaStream_t s) {
  FE_ARG(V.nv >= 0 && V.nv <= kMaxBlocks, "update_gram: nv = %d", V.nv);
  FE_ARG(V.nv == 0 || (V.bv == b && V.ld == b), "update_gram: blocks must be n x b");
#define UG(T, B) return launch_update_gram<T, B, B>(V, n, C, alpha, beta, M, static_cast<T*>(W), gram_v, skip, G, s)
  if (dt == FE_F32) {
    switch (b) { case 1: UG(float, 1); case 2: UG(float, 2); case 4: UG(float, 4); case 8: UG(float, 8); }
  } else {
    switch (b) { case 1: UG(double, 1); case 2: UG(double, 2); case 4: UG(double, 4); case 8: UG(double, 8); }
  }
#undef UG
  return set_error(FE_ERR_INVALID, "update_gram: b = %d not in {1, 2, 4, 8}", b);
}

}  // namespace fe
