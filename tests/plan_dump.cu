// Test helper (host code only, no device work): builds the SpMM plan of a CSR row range with the
// library's own host plan builder (fe::build_host_plan, the degree binning done at handle
// creation) and writes every field of it to a binary file, for tests/test_spmm_plan.py to check
// against the CSR on the CPU.
//
// usage: plan_dump <input> <output>
// input  (little-endian): int64 n, r0, r1; int32 tail_max, hub_min, hub_chunk, packed;
//                         int64 rowptr[n + 1]; int32 colidx[rowptr[n]]
// output: int32 rc, then (rc == 0) int64 scalars max_degree, rows_empty, rows_tail, rows_mid,
//         rows_hub, nbuckets, nslices, ell_total, ntasks, nhub_tasks, nhub, packed; then the
//         arrays deg_of_bucket, deg_slice_begin, deg_ell_base (nbuckets each), slice_rows, ell,
//         hub_rows, hub_task_begin, and either tasks (start, row, len) + tcol or
//         ptasks (woff, row, len, base, w) + tbits -- every array preceded by its int64 length.
#include <cstdio>
#include <vector>

#include "fe_internal.cuh"

template <typename T>
static bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

template <typename T>
static void wr_arr(FILE* f, const T* p, int64_t n) {
  fwrite(&n, sizeof(n), 1, f);
  if (n > 0) fwrite(p, sizeof(T), (size_t)n, f);
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* in = fopen(argv[1], "rb");
  if (!in) return 2;
  int64_t hdr[3];
  int32_t opt[4];
  if (!rd(in, hdr, 3) || !rd(in, opt, 4)) return 2;
  const int64_t n = hdr[0];
  std::vector<int64_t> rowptr(n + 1);
  if (!rd(in, rowptr.data(), n + 1)) return 2;
  std::vector<int32_t> colidx(rowptr[n] > 0 ? rowptr[n] : 1);
  if (rowptr[n] > 0 && !rd(in, colidx.data(), rowptr[n])) return 2;
  fclose(in);

  fe::HostPlan hp;
  const int32_t rc = fe::build_host_plan(rowptr.data(), colidx.data(), hdr[1], hdr[2], opt[0], opt[1],
                                         opt[2], opt[3] != 0, hp);
  FILE* out = fopen(argv[2], "wb");
  if (!out) return 2;
  fwrite(&rc, sizeof(rc), 1, out);
  if (rc == 0) {
    const int64_t sc[12] = {hp.max_degree, hp.rows_empty, hp.rows_tail, hp.rows_mid, hp.rows_hub,
                            hp.nbuckets, hp.nslices, hp.ell_total, hp.ntasks, hp.nhub_tasks,
                            hp.nhub, hp.packed ? 1 : 0};
    fwrite(sc, sizeof(int64_t), 12, out);
    wr_arr(out, hp.deg_of_bucket, hp.nbuckets);
    wr_arr(out, hp.deg_slice_begin, hp.nbuckets);
    wr_arr(out, hp.deg_ell_base, hp.nbuckets);
    wr_arr(out, hp.slice_rows.data(), (int64_t)hp.slice_rows.size());
    wr_arr(out, hp.ell.data(), (int64_t)hp.ell.size());
    wr_arr(out, hp.hub_rows.data(), (int64_t)hp.hub_rows.size());
    wr_arr(out, hp.hub_task_begin.data(), (int64_t)hp.hub_task_begin.size());
    if (!hp.packed) {
      std::vector<int64_t> t(3 * hp.tasks.size());
      for (size_t i = 0; i < hp.tasks.size(); ++i) {
        t[3 * i] = hp.tasks[i].start;
        t[3 * i + 1] = hp.tasks[i].row;
        t[3 * i + 2] = hp.tasks[i].len;
      }
      wr_arr(out, t.data(), (int64_t)t.size());
      wr_arr(out, hp.tcol.data(), (int64_t)hp.tcol.size());
    } else {
      std::vector<int64_t> t(5 * hp.ptasks.size());
      for (size_t i = 0; i < hp.ptasks.size(); ++i) {
        const fe::PTask& p = hp.ptasks[i];
        t[5 * i] = p.woff;
        t[5 * i + 1] = p.row;
        t[5 * i + 2] = p.len;
        t[5 * i + 3] = p.base;
        t[5 * i + 4] = p.w;
      }
      wr_arr(out, t.data(), (int64_t)t.size());
      wr_arr(out, hp.tbits.data(), (int64_t)hp.tbits.size());
    }
  }
  fclose(out);
  return 0;
}
