// Rayleigh-Ritz on the projected matrix (Algorithm 1 steps (2)-(4)) and the Krylov-Schur
// restart of the small matrix, on the device.
//
// ritz_kernel: T = (H_m + H_m^T) / 2 (m x m) is diagonalised by the cyclic Jacobi method in
// parallel ("round-robin" ordering, Brent & Luk 1985: each of the m-1 steps of a sweep
// rotates m/2 disjoint index pairs at once, so the row and column updates of different pairs
// never touch the same entries).  Each rotation is the 2x2 symmetric Schur decomposition of
// Golub & Van Loan Section 8.5.  The Ritz values are then ordered by `which`, and each Ritz
// pair gets its residual estimate rho_c = ||H[m:m+b, 0:m] y_c|| (the coupling of the last
// block to the next basis block, since A V_m = V_m H_m + V_{NB} H[m:m+b, :]).
#include <math.h>

#include "fe_internal.cuh"

namespace fe {

// smem layout: A[mp][mp+1], Q[mp][mp+1] (padded rows), plus pair rotations.
__global__ void ritz_kernel(const double* __restrict__ H, int m, int b, int which, int max_sweeps,
                            double tol, double* __restrict__ theta_out, double* __restrict__ Y_out,
                            double* __restrict__ rho_out, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int mp = m + (m & 1);  // even size; index m (if odd) is a zero dummy never rotated
  const int ld = mp + 1;
  double* A = reinterpret_cast<double*>(smem_raw);
  double* Q = A + (size_t)mp * ld;
  double* cs = Q + (size_t)mp * ld;
  double* sn = cs + mp / 2;
  int* pp = reinterpret_cast<int*>(sn + mp / 2);
  int* pq = pp + mp / 2;
  int* order = pq + mp / 2;
  __shared__ double red[32];
  __shared__ double fro2;
  __shared__ int done;
  const int tid = threadIdx.x, nth = blockDim.x;

  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    double a = 0.0;
    if (i < m && j < m) a = 0.5 * (H[i * m + j] + H[j * m + i]);
    A[i * ld + j] = a;
    Q[i * ld + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  auto block_sum = [&](double v) -> double {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0) {
      for (int w = 0; w < (nth + 31) / 32; ++w) s += red[w];
      red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
  };
  {
    double v = 0.0;
    for (int e = tid; e < mp * mp; e += nth) v += A[(e / mp) * ld + e % mp] * A[(e / mp) * ld + e % mp];
    double s = block_sum(v);
    if (tid == 0) fro2 = s;
  }
  __syncthreads();
  int sweeps = 0;
  bool converged = false;
  while (true) {
    double v = 0.0;
    for (int e = tid; e < mp * mp; e += nth) {
      const int i = e / mp, j = e % mp;
      if (i != j) v += A[i * ld + j] * A[i * ld + j];
    }
    const double off2 = block_sum(v);
    if (tid == 0) done = (off2 <= tol * tol * fro2) || sweeps >= max_sweeps;
    __syncthreads();
    if (done) {
      converged = off2 <= tol * tol * fro2;
      break;
    }
    ++sweeps;
    for (int step = 0; step < mp - 1; ++step) {
      // circle method: position 0 fixed, positions 1..mp-1 rotate by `step`
      for (int k = tid; k < mp / 2; k += nth) {
        auto pos = [&](int i) { return i == 0 ? 0 : ((i - 1 + step) % (mp - 1)) + 1; };
        int p = pos(k), q = pos(mp - 1 - k);
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p * ld + q];
          if (apq != 0.0) {
            const double tau = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pp[k] = p;
        pq[k] = q;
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      // rows p, q  (A <- J^T A)
      for (int e = tid; e < (mp / 2) * mp; e += nth) {
        const int k = e / mp, j = e % mp;
        const double c = cs[k], s = sn[k];
        if (s == 0.0) continue;
        const int p = pp[k], q = pq[k];
        const double ap = A[p * ld + j], aq = A[q * ld + j];
        A[p * ld + j] = c * ap - s * aq;
        A[q * ld + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q  (A <- A J, Q <- Q J)
      for (int e = tid; e < (mp / 2) * mp; e += nth) {
        const int k = e / mp, i = e % mp;
        const double c = cs[k], s = sn[k];
        if (s == 0.0) continue;
        const int p = pp[k], q = pq[k];
        const double ap = A[i * ld + p], aq = A[i * ld + q];
        A[i * ld + p] = c * ap - s * aq;
        A[i * ld + q] = s * ap + c * aq;
        const double vp = Q[i * ld + p], vq = Q[i * ld + q];
        Q[i * ld + p] = c * vp - s * vq;
        Q[i * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // order by `which` (stable insertion sort; 0 = LM: |x| desc, ties larger first;
  // 1 = LA: descending; 2 = SA: ascending)
  if (tid == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 1; i < m; ++i) {
      const int x = order[i];
      const double tx = A[x * ld + x];
      int j = i - 1;
      while (j >= 0) {
        const double ty = A[order[j] * ld + order[j]];
        bool before;
        if (which == 0) before = fabs(tx) > fabs(ty) || (fabs(tx) == fabs(ty) && tx > ty);
        else if (which == 1) before = tx > ty;
        else before = tx < ty;
        if (!before) break;
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = x;
    }
    info[0] = converged ? sweeps : -1;
  }
  __syncthreads();
  for (int c = tid; c < m; c += nth) theta_out[c] = A[order[c] * ld + order[c]];
  for (int e = tid; e < m * m; e += nth) {
    const int i = e / m, c = e % m;
    Y_out[e] = Q[i * ld + order[c]];
  }
  for (int c = tid; c < m; c += nth) {
    double r2 = 0.0;
    for (int p = 0; p < b; ++p) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += H[(m + p) * m + i] * Q[i * ld + order[c]];
      r2 += s * s;
    }
    rho_out[c] = sqrt(r2);
  }
}

size_t ritz_smem_bytes(int m) {
  const int mp = m + (m & 1);
  return (size_t)2 * mp * (mp + 1) * sizeof(double) + (size_t)mp * sizeof(double) +
         (size_t)(mp / 2) * 2 * sizeof(int) + (size_t)mp * sizeof(int) + 64;
}

int launch_ritz(const double* H, int m, int b, int which, int max_sweeps, double tol,
                double* theta, double* Y, double* rho, int* info, cudaStream_t s) {
  const size_t smem = ritz_smem_bytes(m);
  FE_ARG(smem <= 220 * 1024, "ritz: subspace m = %d too large", m);
  static bool configured = false;
  if (!configured) {
    FE_CUDA(cudaFuncSetAttribute(ritz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    configured = true;
  }
  // few threads: each of the ~3 barriers per rotation step is cheap, and a step is only
  // m/2 x m updates
  ritz_kernel<<<1, 128, smem, s>>>(H, m, b, which, max_sweeps, tol, theta, Y, rho, info);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// Krylov-Schur restart of H ((m+b) x m, row-major): keep k Ritz pairs.
//   B^T = H[m:m+b, 0:m] Y[:, 0:k];  H <- 0;  H[c][c] = theta_c (c < k);  H[k:k+b, 0:k] = B^T
__global__ void restart_h_kernel(double* __restrict__ H, int m, int b, int k,
                                 const double* __restrict__ theta, const double* __restrict__ Y) {
  extern __shared__ double bt[];  // b x k
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < b * k; e += nth) {
    const int p = e / k, c = e % k;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += H[(m + p) * m + i] * Y[i * m + c];
    bt[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < (m + b) * m; e += nth) H[e] = 0.0;
  __syncthreads();
  for (int c = tid; c < k; c += nth) H[c * m + c] = theta[c];
  for (int e = tid; e < b * k; e += nth) H[(k + e / k) * m + e % k] = bt[e];
}

int launch_restart_h(double* H, int m, int b, int k, const double* theta, const double* Y,
                     cudaStream_t s) {
  restart_h_kernel<<<1, 256, sizeof(double) * b * k, s>>>(H, m, b, k, theta, Y);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// ------------------------------------------------------------ sign of eigenvectors
// For each column c of the column-major n x ncols matrix X: find the entry of largest
// magnitude (first index on ties) and flip the column if it is negative.  The partials carry
// the signed value of each block's best entry, so the flip decision never re-reads X (which
// other blocks of the flipping kernel may already have changed).
__global__ void colmax_partial_kernel(const double* __restrict__ X, int64_t n, int ncols,
                                      double* __restrict__ pval, int64_t* __restrict__ pidx) {
  const int c = blockIdx.y;
  double best = -1.0, bval = 0.0;
  int64_t bi = INT64_MAX;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[(int64_t)c * n + r];
    const double a = fabs(x);
    if (a > best || (a == best && r < bi)) { best = a; bi = r; bval = x; }
  }
  __shared__ double sv[256], sx[256];
  __shared__ int64_t si[256];
  sv[threadIdx.x] = best;
  sx[threadIdx.x] = bval;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double a = sv[threadIdx.x + w];
      const int64_t i = si[threadIdx.x + w];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && i < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = i;
        sx[threadIdx.x] = sx[threadIdx.x + w];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pval[(int64_t)c * gridDim.x + blockIdx.x] = sx[0];   // signed value of the best entry
    pidx[(int64_t)c * gridDim.x + blockIdx.x] = si[0];
  }
}

__global__ void colsign_kernel(double* __restrict__ X, int64_t n, int ncols, int nparts,
                               const double* __restrict__ pval, const int64_t* __restrict__ pidx) {
  const int c = blockIdx.y;
  __shared__ double sgn;
  if (threadIdx.x == 0) {
    double best = -1.0, bval = 0.0;
    int64_t bi = INT64_MAX;
    for (int p = 0; p < nparts; ++p) {
      const double x = pval[(int64_t)c * nparts + p];
      const double a = fabs(x);
      const int64_t i = pidx[(int64_t)c * nparts + p];
      if (a > best || (a == best && i < bi)) { best = a; bi = i; bval = x; }
    }
    sgn = bval < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  if (sgn > 0.0) return;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)c * n + r] = -X[(int64_t)c * n + r];
}

int normalize_signs(double* X, int64_t n, int ncols, cudaStream_t s) {
  const int parts = (int)std::min<int64_t>(ceil_div(n, 256), 64);
  double* pval = small_scratch(12, (size_t)parts * ncols);
  double* pidx = small_scratch(13, (size_t)parts * ncols);
  if (!pval || !pidx) return FE_ERR_OOM;
  dim3 grid(parts, ncols);
  colmax_partial_kernel<<<grid, 256, 0, s>>>(X, n, ncols, pval, reinterpret_cast<int64_t*>(pidx));
  count_launch();
  FE_CUDA(cudaGetLastError());
  colsign_kernel<<<grid, 256, 0, s>>>(X, n, ncols, parts, pval, reinterpret_cast<const int64_t*>(pidx));
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

}  // namespace fe
