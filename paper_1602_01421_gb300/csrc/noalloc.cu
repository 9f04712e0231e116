// fe_block_gram_noalloc: the Gram product V^T W for callers that must not allocate device
// memory.  The per-CTA partial sums, which fe_block_gram keeps in a buffer it allocates on
// demand, live here in a fixed file-scope device array instead.
#include <mutex>

#include "fe_internal.cuh"

namespace fe {

int gram_into_scratch(const BlockSet& V, int64_t n, const void* W, int bw, int ldw, fe_dtype dt,
                      double alpha, double* G, double* scratch, size_t capacity, cudaStream_t s);

// 2 MiB of partial sums.  Every device that loads the library holds this array until the
// process exits.
constexpr size_t kNoAllocScratchDoubles = 262144;
constexpr int kNoAllocMaxOutputs = 2048;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

static double* g_noalloc_addr[kMaxDevices];  // device address of the array, per device
static std::mutex g_noalloc_mu;

// In host code g_noalloc_scratch names a host-side stand-in, not device memory, so the
// array's device address is looked up once per device (with that device current) and kept.
static int noalloc_scratch_address(double** out) {
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev));
  FE_ARG(dev >= 0 && dev < kMaxDevices, "fe_block_gram_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" int fe_block_gram_noalloc(const void* V, int64_t n, int nv, int bv, const void* W,
                                     int bw, fe_dtype dt, double alpha, double* G) {
  FE_ARG(V && W && G, "fe_block_gram_noalloc: NULL pointer");
  FE_ARG(n >= 1, "fe_block_gram_noalloc: n < 1");
  FE_ARG(nv >= 1 && nv <= 32, "fe_block_gram_noalloc: nv = %d not in [1, 32]", nv);
  FE_ARG(is_pow2_le16(bv) && is_pow2_le16(bw), "fe_block_gram_noalloc: bv, bw must be in {1,2,4,8,16}");
  FE_ARG(dt == FE_F32 || dt == FE_F64, "fe_block_gram_noalloc: bad dtype");
  FE_ARG(aligned16(V) && aligned16(W), "fe_block_gram_noalloc: V and W must be 16-byte aligned");
  const int nout = nv * bv * bw;
  FE_ARG(nout <= kNoAllocMaxOutputs,
         "fe_block_gram_noalloc: G has nv*bv*bw = %d entries, more than the %d this entry point "
         "supports (its static scratch is %zu doubles); use fe_block_gram",
         nout, kNoAllocMaxOutputs, kNoAllocScratchDoubles);
  double* scratch = nullptr;
  FE_TRY(noalloc_scratch_address(&scratch));
  BlockSet vs = make_blockset(V, nv, bv, bv, n * bv, dt);
  return gram_into_scratch(vs, n, W, bw, bw, dt, alpha, G, scratch, kNoAllocScratchDoubles,
                           cur_stream());
}
