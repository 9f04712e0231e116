// Rayleigh-Ritz on the projected matrix (Algorithm 1 steps (2)-(4)) and the Krylov-Schur
// restart of the small matrix, on the device.
//
// ritz_kernel: T = (H_m + H_m^T) / 2 (m x m) is diagonalised by the cyclic Jacobi method in
// parallel ("round-robin" ordering, Brent & Luk 1985: each of the m-1 steps of a sweep
// rotates m/2 disjoint index pairs at once).  Each rotation is the 2x2 symmetric Schur
// decomposition of Golub & Van Loan Section 8.5; a step applies all of them at once as
// J^T A J on independent 2x2 blocks (rows of one pair, columns of another), so a step costs
// two barriers.  The Ritz values are then ordered by `which`, and each Ritz
// pair gets its residual estimate rho_c = ||H[m:m+b, 0:m] y_c|| (the coupling of the last
// block to the next basis block, since A V_m = V_m H_m + V_{NB} H[m:m+b, :]).
#include <math.h>

#include "fe_internal.cuh"

namespace fe {

// tan of the Jacobi angle that diagonalises [app apq; apq aqq] (Golub & Van Loan Section
// 8.5.2), evaluated in FP32.  FP64 entries are first scaled by a power of two and the diagonal
// difference is taken in FP64, so only the final quotient and square root are FP32.  Returns
// 0 when apq is negligible at FP32 range.  Any t gives an exactly orthogonal rotation once c
// and s are formed from it (jacobi_cs), so an inexact t only leaves a small (p,q) entry for
// the next sweep.
__device__ __forceinline__ float jacobi_tan(float app, float apq, float aqq) {
  if (apq == 0.f) return 0.f;
  const float tau = (aqq - app) / (2.f * apq);
  if (fabsf(tau) > 1e18f) return 0.5f / tau;
  return (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
}
__device__ __forceinline__ float jacobi_tan(double app, double apq, double aqq) {
  if (apq == 0.0) return 0.f;
  const double mx = fmax(fmax(fabs(app), fabs(aqq)), fabs(apq));
  int e;
  frexp(mx, &e);
  const double sc = ldexp(1.0, -e);
  const float d = (float)((aqq - app) * sc), f = (float)(apq * sc);
  if (f == 0.f) return 0.f;
  const float tau = d / (2.f * f);
  if (fabsf(tau) > 1e18f) return 0.5f / tau;
  return (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
}
// c = 1 / sqrt(1 + t^2), s = t c in T: FP32 estimate, then (FP64) two Newton steps for the
// reciprocal square root, so that c^2 + s^2 = 1 to T's rounding.
__device__ __forceinline__ void jacobi_cs(float t, float& c, float& s) {
  c = rsqrtf(1.f + t * t);
  s = t * c;
}
__device__ __forceinline__ void jacobi_cs(float t32, double& c, double& s) {
  const double t = (double)t32, u = 1.0 + t * t;
  double r = (double)rsqrtf((float)u);
  r = r * (1.5 - 0.5 * u * r * r);
  r = r * (1.5 - 0.5 * u * r * r);
  c = r;
  s = t * r;
}

// Sum over the block of one value per thread (all threads call it).
__device__ double ritz_block_sum(double v, double* red) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (nth + 31) / 32; ++w) s += red[w];
    red[0] = s;
  }
  __syncthreads();
  const double s = red[0];
  __syncthreads();
  return s;
}

// Parallel cyclic Jacobi sweeps on the symmetric mp x mp matrix A (row stride ld), with
// Q <- Q J accumulated, until the off-diagonal Frobenius norm squared is <= thresh or after
// max_sweeps.  Returns the sweeps run; *conv tells whether the threshold was met.
template <typename T>
__device__ int jacobi_sweeps(T* A, T* Q, int ld, int m, int mp, double thresh, int max_sweeps,
                             T* cs, T* sn, int* pp, int* pq, double* red, bool* conv) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int np = mp / 2;
  int sweeps = 0;
  while (true) {
    double v = 0.0;
    for (int e = tid; e < mp * mp; e += nth) {
      const int i = e / mp, j = e - (e / mp) * mp;
      if (i != j) v += (double)A[i * ld + j] * (double)A[i * ld + j];
    }
    const double off2 = ritz_block_sum(v, red);
    if (off2 <= thresh || sweeps >= max_sweeps) {
      *conv = off2 <= thresh;
      return sweeps;
    }
    ++sweeps;
    for (int step = 0; step < mp - 1; ++step) {
      // circle method: position 0 fixed, positions 1..mp-1 rotate by `step`
      for (int k = tid; k < np; k += nth) {
        auto pos = [&](int i) { return i == 0 ? 0 : ((i - 1 + step) % (mp - 1)) + 1; };
        int p = pos(k), q = pos(mp - 1 - k);
        if (p > q) { int t = p; p = q; q = t; }
        T c = T(1), sv = T(0);
        if (q < m) {
          const float t = jacobi_tan(A[p * ld + p], A[p * ld + q], A[q * ld + q]);
          if (t != 0.f) jacobi_cs(t, c, sv);
        }
        pp[k] = p;
        pq[k] = q;
        cs[k] = c;
        sn[k] = sv;
      }
      __syncthreads();
      // A <- J^T A J as independent 2 x 2 blocks (rows of pair k, columns of pair k2, k <= k2,
      // mirrored to the lower triangle), and Q <- Q J by column pairs: the step's pairs are
      // disjoint, so no two work items touch the same entry and one barrier suffices.
      const int nsq = np * np;
      for (int e = tid; e < nsq + mp * np; e += nth) {
        if (e < nsq) {
          const int k = e / np, k2 = e - k * np;
          if (k > k2) continue;
          const T s1 = sn[k], s2 = sn[k2];
          if (s1 == T(0) && s2 == T(0)) continue;
          const T c1 = cs[k], c2 = cs[k2];
          const int p1 = pp[k], q1 = pq[k];
          if (k == k2) {
            // the pair's own block: full transform (t need not be exact)
            const T app = A[p1 * ld + p1], aqq = A[q1 * ld + q1], apq = A[p1 * ld + q1];
            const T cc = c1 * c1, ss = s1 * s1, cs2 = c1 * s1;
            A[p1 * ld + p1] = cc * app - T(2) * cs2 * apq + ss * aqq;
            A[q1 * ld + q1] = ss * app + T(2) * cs2 * apq + cc * aqq;
            const T npq = cs2 * (app - aqq) + (cc - ss) * apq;
            A[p1 * ld + q1] = npq;
            A[q1 * ld + p1] = npq;
          } else {
            const int p2 = pp[k2], q2 = pq[k2];
            const T x00 = A[p1 * ld + p2], x01 = A[p1 * ld + q2];
            const T x10 = A[q1 * ld + p2], x11 = A[q1 * ld + q2];
            const T y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
            const T y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
            const T z00 = c2 * y00 - s2 * y01, z01 = s2 * y00 + c2 * y01;
            const T z10 = c2 * y10 - s2 * y11, z11 = s2 * y10 + c2 * y11;
            A[p1 * ld + p2] = z00;
            A[p1 * ld + q2] = z01;
            A[q1 * ld + p2] = z10;
            A[q1 * ld + q2] = z11;
            A[p2 * ld + p1] = z00;
            A[q2 * ld + p1] = z01;
            A[p2 * ld + q1] = z10;
            A[q2 * ld + q1] = z11;
          }
        } else {
          const int e2 = e - nsq;
          const int i = e2 / np, k = e2 - i * np;
          const T sk = sn[k];
          if (sk == T(0)) continue;
          const T ck = cs[k];
          const int p = pp[k], q = pq[k];
          const T vp = Q[i * ld + p], vq = Q[i * ld + q];
          Q[i * ld + p] = ck * vp - sk * vq;
          Q[i * ld + q] = sk * vp + ck * vq;
        }
      }
      __syncthreads();
    }
  }
}

// smem layout (mp = m rounded up to even, ld = mp + 1, rows padded), m <= kRitzSmallMax:
//   A64[mp][ld], Q64[mp][ld]             FP64 matrix and eigenvectors
//   U: A32[mp][ld] + Q32[mp][ld] (FP32)  later reused as W[mp][ld] (FP64 scratch)
//   cs, sn (mp/2 doubles each), pp, pq (mp/2 ints each), order (mp ints)
// Larger subspaces (BIG, m <= kRitzMax): the FP32 pair A32 + Q32 occupies the A64 region and
// A64 is rebuilt from H once the FP32 sweeps are done; Q64 and W live in `gwork`
// (2 mp ld doubles of global memory, L2-resident).
// Two precisions: FP32 Jacobi sweeps take the matrix to a relative off-diagonal norm of about
// 1e-6 (FP32 rotations run at the FP32 rate of the SM, FP64 ones at 1/64 of it); the FP32
// eigenvector matrix is made exactly orthogonal in FP64 (Cholesky QR), the FP64 matrix is
// transformed by it (Q^T T Q, an exact orthogonal similarity), and FP64 sweeps finish from there
// -- two or three, since Jacobi converges quadratically once the off-diagonal part is small.
template <bool BIG>
__global__ void ritz_kernel(const double* __restrict__ H, int m, int b, int which, int max_sweeps,
                            double tol, double* __restrict__ theta_out, double* __restrict__ Y_out,
                            double* __restrict__ rho_out, int* __restrict__ info, double* gwork) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int mp = m + (m & 1);  // even size; index m (if odd) is a zero dummy never rotated
  const int ld = mp + 1;
  const size_t mat = (size_t)mp * ld;
  double* A = reinterpret_cast<double*>(smem_raw);
  double* Q = BIG ? gwork : A + mat;
  double* W = BIG ? gwork + mat : Q + mat;
  float* A32 = BIG ? reinterpret_cast<float*>(A) : reinterpret_cast<float*>(W);
  float* Q32 = A32 + mat;
  const int np = mp / 2;  // rotation pairs per step
  double* cs = BIG ? A + mat : W + mat;
  double* sn = cs + np;
  int* pp = reinterpret_cast<int*>(sn + np);
  int* pq = pp + np;
  int* order = pq + np;
  __shared__ double red[32];
  __shared__ bool conv32, conv64;
  const int tid = threadIdx.x, nth = blockDim.x;

  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    double a = 0.0;
    if (i < m && j < m) a = 0.5 * (H[i * m + j] + H[j * m + i]);
    if (!BIG) A[i * ld + j] = a;
    A32[i * ld + j] = (float)a;
    Q32[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  double fro2;
  {
    double v = 0.0;
    for (int e = tid; e < m * m; e += nth) {
      const int i = e / m, j = e % m;
      const double a = 0.5 * (H[i * m + j] + H[j * m + i]);
      v += a * a;
    }
    fro2 = ritz_block_sum(v, red);
  }
  // FP32 sweeps
  int sweeps = jacobi_sweeps<float>(A32, Q32, ld, m, mp, 1e-12 * fro2, 15, reinterpret_cast<float*>(cs),
                                    reinterpret_cast<float*>(sn), pp, pq, red, &conv32);
  // Q = chol-QR(Q32) in FP64: S = Q^T Q (in W after Q32 is copied out), S = R^T R, Q <- Q R^-1
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    Q[i * ld + j] = (double)Q32[i * ld + j];
  }
  __syncthreads();
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    if (i > j) continue;
    double s = 0.0;
    for (int r = 0; r < mp; ++r) s += Q[r * ld + i] * Q[r * ld + j];
    W[i * ld + j] = s;
  }
  __syncthreads();
  for (int j = 0; j < mp; ++j) {
    if (tid == 0) {
      double d = W[j * ld + j];
      for (int l = 0; l < j; ++l) d -= W[l * ld + j] * W[l * ld + j];
      W[j * ld + j] = d > 0.0 ? sqrt(d) : 1.0;  // Q32 is orthogonal to ~1e-7: d ~ 1
    }
    __syncthreads();
    const double rjj = W[j * ld + j];
    for (int i = j + 1 + tid; i < mp; i += nth) {
      double s = W[j * ld + i];
      for (int l = 0; l < j; ++l) s -= W[l * ld + j] * W[l * ld + i];
      W[j * ld + i] = s / rjj;
    }
    __syncthreads();
  }
  for (int r = tid; r < mp; r += nth) {
    for (int j = 0; j < mp; ++j) {
      double x = Q[r * ld + j];
      for (int l = 0; l < j; ++l) x -= Q[r * ld + l] * W[l * ld + j];
      Q[r * ld + j] = x / W[j * ld + j];
    }
  }
  __syncthreads();
  if (BIG) {  // the FP32 pair is dead: A64 takes its region back
    for (int e = tid; e < mp * mp; e += nth) {
      const int i = e / mp, j = e % mp;
      A[i * ld + j] = (i < m && j < m) ? 0.5 * (H[i * m + j] + H[j * m + i]) : 0.0;
    }
    __syncthreads();
  }
  // A <- Q^T A Q (W = A Q first; A is symmetric, the result is mirrored from its upper triangle)
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    double s = 0.0;
    for (int l = 0; l < mp; ++l) s += A[i * ld + l] * Q[l * ld + j];
    W[i * ld + j] = s;
  }
  __syncthreads();
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    if (i > j) continue;
    double s = 0.0;
    for (int l = 0; l < mp; ++l) s += Q[l * ld + i] * W[l * ld + j];
    A[i * ld + j] = s;
    A[j * ld + i] = s;
  }
  __syncthreads();
  // FP64 sweeps to the requested tolerance
  sweeps += jacobi_sweeps<double>(A, Q, ld, m, mp, tol * tol * fro2, max_sweeps, cs, sn, pp, pq,
                                  red, &conv64);
  const bool converged = conv64;
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
  const size_t mats = m <= kRitzSmallMax ? 3 : 1;
  return mats * mp * (mp + 1) * sizeof(double) + (size_t)(mp / 2) * 2 * sizeof(double) +
         (size_t)(mp / 2) * 2 * sizeof(int) + (size_t)mp * sizeof(int) + 64;
}

size_t ritz_work_doubles(int m) {
  const int mp = m + (m & 1);
  return m <= kRitzSmallMax ? 0 : (size_t)2 * mp * (mp + 1);
}

int launch_ritz(const double* H, int m, int b, int which, int max_sweeps, double tol,
                double* theta, double* Y, double* rho, int* info, double* work, cudaStream_t s) {
  const size_t smem = ritz_smem_bytes(m);
  FE_ARG(m >= 1 && m <= kRitzMax, "ritz: subspace m = %d not in [1, %d]", m, kRitzMax);
  FE_ARG(smem <= 225 * 1024, "ritz: subspace m = %d too large", m);
  const bool big = m > kRitzSmallMax;
  FE_ARG(!big || work != nullptr, "ritz: m = %d needs a global workspace", m);
  static KernelSetup ks[2];
  FE_TRY(kernel_configure(ks[big], big ? reinterpret_cast<const void*>(ritz_kernel<true>)
                                       : reinterpret_cast<const void*>(ritz_kernel<false>),
                          225 * 1024));
  // one CTA: a rotation step is (m/2)^2 / 2 2 x 2 blocks plus m^2 / 2 Q updates between two
  // barriers; FP64 work on one SM runs at 2 DFMA per clock, hence the FP32 sweeps first
  if (big)
    ritz_kernel<true><<<1, 512, smem, s>>>(H, m, b, which, max_sweeps, tol, theta, Y, rho, info, work);
  else
    ritz_kernel<false><<<1, 256, smem, s>>>(H, m, b, which, max_sweeps, tol, theta, Y, rho, info, nullptr);
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
