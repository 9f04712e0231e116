// Row partition of the sparse matrix for a multi-GPU layout (host code).  The paper runs its
// eigensolver on one machine (Section 3); split over several GPUs, the method shards by rows:
// each part owns a contiguous row range of A and of every n x b block, an SpMM needs the X rows
// its part's column indices reference (an all-gather of X, or only the halo rows), and the
// Gram products V^T W are sums of per-part partial products (an all-reduce of the small
// result).  These functions compute the partition and one part's local CSR; the exchange
// itself is the caller's (the Python package's dist module, over torch.distributed).
#include <string.h>

#include <algorithm>
#include <vector>

#include "fe_internal.cuh"

using namespace fe;

extern "C" {

int fe_partition_rows(int64_t n, const int64_t* rowptr, int nparts, int64_t* row_begin) {
  FE_ARG(rowptr && row_begin, "fe_partition_rows: NULL pointer");
  FE_ARG(n >= 1, "fe_partition_rows: n < 1");
  FE_ARG(nparts >= 1 && nparts <= 65536, "fe_partition_rows: nparts = %d", nparts);
  FE_ARG(rowptr[0] == 0, "fe_partition_rows: rowptr[0] != 0");
  for (int64_t i = 0; i < n; ++i)
    FE_ARG(rowptr[i + 1] >= rowptr[i], "fe_partition_rows: rowptr decreases at row %lld", (long long)i);
  // cost of rows [0, i) = rowptr[i] + i: every non-zero is one gather, every row one output
  const int64_t total = rowptr[n] + n;
  row_begin[0] = 0;
  for (int p = 1; p < nparts; ++p) {
    const int64_t target = (total * p) / nparts;
    // smallest i with cost(i) >= target, searched between the previous boundary and n
    int64_t lo = row_begin[p - 1], hi = n;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (rowptr[mid] + mid >= target) hi = mid;
      else lo = mid + 1;
    }
    row_begin[p] = lo;
  }
  row_begin[nparts] = n;
  return FE_OK;
}

int fe_partition_local(int64_t n, const int64_t* rowptr, const int32_t* colidx, int64_t r0, int64_t r1,
                       int64_t* local_rowptr, int32_t* local_colidx, int32_t* halo, int64_t* nhalo) {
  FE_ARG(rowptr && colidx && local_rowptr && nhalo, "fe_partition_local: NULL pointer");
  FE_ARG(n >= 1 && 0 <= r0 && r0 <= r1 && r1 <= n, "fe_partition_local: bad row range [%lld, %lld)",
         (long long)r0, (long long)r1);
  const int64_t base = rowptr[r0];
  const int64_t nnz = rowptr[r1] - base;
  FE_ARG(nnz == 0 || local_colidx, "fe_partition_local: NULL local_colidx");
  for (int64_t i = r0; i <= r1; ++i) local_rowptr[i - r0] = rowptr[i] - base;
  std::vector<int32_t> ext;
  for (int64_t k = 0; k < nnz; ++k) {
    const int32_t c = colidx[base + k];
    FE_ARG(c >= 0 && c < n, "fe_partition_local: column %d out of range", c);
    local_colidx[k] = c;
    if (c < r0 || c >= r1) ext.push_back(c);
  }
  std::sort(ext.begin(), ext.end());
  ext.erase(std::unique(ext.begin(), ext.end()), ext.end());
  *nhalo = (int64_t)ext.size();
  if (halo && !ext.empty()) memcpy(halo, ext.data(), sizeof(int32_t) * ext.size());
  return FE_OK;
}

}  // extern "C"
