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

#include <algorithm>

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

// e / d for 0 <= e < 2^22 and 1 <= d < 2^11, with inv = 1 / d: an FP32 estimate corrected once
// (an integer division would be a long instruction sequence inside the work loops).
__device__ __forceinline__ int small_div(int e, int d, float inv) {
  int q = (int)((float)e * inv);
  const int r = e - q * d;
  q += r < 0 ? -1 : (r >= d ? 1 : 0);
  return q;
}

// The e-th of the pairs (k, k2), k <= k2 < np (the upper triangle of the step's 2 x 2 blocks,
// np (np + 1) / 2 of them), from a triangular-number inversion in FP32 corrected in integers.
__device__ __forceinline__ void tri_pair(int e, int np, int& k, int& k2) {
  const int f = np * (np + 1) / 2 - 1 - e;   // reversed index: row r holds r + 1 items
  int r = (int)((sqrtf(8.f * (float)f + 1.f) - 1.f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= f) ++r;
  if (r * (r + 1) / 2 > f) --r;
  const int o = f - r * (r + 1) / 2;
  k = np - 1 - r;
  k2 = np - 1 - o;
}

// Parallel cyclic Jacobi sweeps on the symmetric mp x mp matrix A (row stride ld), with
// Q <- Q J accumulated, until the off-diagonal Frobenius norm squared is <= thresh or after
// max_sweeps.  Returns the sweeps run; *conv tells whether the threshold was met.
template <typename T>
__device__ int jacobi_sweeps(T* A, T* Q, int ld, int m, int mp, double thresh, int max_sweeps,
                             T* cs, T* sn, int* pp, int* pq, double* red, bool* conv) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int np = mp / 2;
  const float inv_mp = 1.f / (float)mp, inv_np = 1.f / (float)np;
  const int ntri = np * (np + 1) / 2;
  int sweeps = 0;
  while (true) {
    double v = 0.0;
    for (int e = tid; e < mp * mp; e += nth) {
      const int i = small_div(e, mp, inv_mp), j = e - i * mp;
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
      for (int e = tid; e < ntri + mp * np; e += nth) {
        if (e < ntri) {
          int k, k2;
          tri_pair(e, np, k, k2);
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
          const int e2 = e - ntri;
          const int i = small_div(e2, np, inv_np), k = e2 - i * np;
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
// eigenvector matrix is made orthogonal to FP64 rounding (two Newton-Schulz steps), the FP64 matrix is
// transformed by it (Q^T T Q, an exact orthogonal similarity), and FP64 sweeps finish from there
// -- two or three, since Jacobi converges quadratically once the off-diagonal part is small.
template <bool BIG>
__global__ void __launch_bounds__(1024) ritz_kernel(const double* __restrict__ H, int m, int b, int which, int max_sweeps,
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
  // Q32 made orthogonal in FP64 by two Newton-Schulz steps Q <- Q (3 I - Q^T Q) / 2 (Higham,
  // "Functions of Matrices", 8.3: quadratic convergence to the orthogonal polar factor from
  // ||Q^T Q - I|| ~ 1e-6, to FP64 rounding in two steps); S and the factor in W, each new row
  // of Q formed by one warp (all of its entries read before any is written)
  const float inv_mp = 1.f / (float)mp;
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = small_div(e, mp, inv_mp), j = e - i * mp;
    Q[i * ld + j] = (double)Q32[i * ld + j];
  }
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    for (int e = tid; e < mp * mp; e += nth) {
      const int i = small_div(e, mp, inv_mp), j = e - i * mp;
      if (i > j) continue;
      double sv = 0.0;
      for (int r = 0; r < mp; ++r) sv = fma(Q[r * ld + i], Q[r * ld + j], sv);
      const double f = (i == j ? 1.5 : 0.0) - 0.5 * sv;
      W[i * ld + j] = f;
      W[j * ld + i] = f;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
    for (int r = warp; r < mp; r += nwarps) {
      double x[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // columns lane + 32 t (mp <= 160)
      for (int l = 0; l < mp; ++l) {
        const double q = Q[r * ld + l];
#pragma unroll
        for (int t = 0; t < 5; ++t)
          if (lane + 32 * t < mp) x[t] = fma(q, W[l * ld + lane + 32 * t], x[t]);
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 5; ++t)
        if (lane + 32 * t < mp) Q[r * ld + lane + 32 * t] = x[t];
    }
    __syncthreads();
  }
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

// ------------------------------------------------------------ large subspaces (m > kRitzMidMax)
// For m up to kRitzMax (512) the m x m matrices no longer fit one SM's shared memory, and FP64
// Jacobi work on one SM (2 DFMA per clock) would take tens of milliseconds per sweep.  So:
//   1. one CTA runs the FP32 Jacobi sweeps (A32, Q32 in global memory, L2-resident) to a
//      relative off-diagonal norm of about 1e-6;
//   2. Q32 is made orthogonal in FP64 by two Newton-Schulz steps Q <- Q (3 I - Q^T Q) / 2
//      (Higham, "Functions of Matrices", 8.3: quadratic convergence to the orthogonal polar
//      factor from ||Q^T Q - I|| ~ 1e-7), and A <- Q^T T Q, all as FP64 matrix products on the
//      whole GPU;
//   3. FP64 parallel Jacobi sweeps on the nearly diagonal A finish it (two or three sweeps), on
//      a cooperative grid: a step's rotations are computed by every CTA from the same entries,
//      then the CTAs share the step's 2 x 2 block updates, with a grid barrier after each half;
//   4. one CTA orders the pairs and writes theta, Y and the residual estimates.
// Workspace layout (ld = mp + 1): A32, Q32 (floats, one mp x ld double-array each pair), A64,
// Q64, W64, S64, then the barrier words and the per-CTA partial sums.
constexpr int kRitzMidMax = 160;   // the one-CTA kernel's limit (global FP64 Q above 96)
constexpr int kCoopCtas = 64;

struct BigWork {
  float *A32, *Q32;
  double *A, *Q, *W, *S;
  unsigned* bar;      // [0] arrivals, [1] generation, [2] error flag
  double* part;       // kCoopCtas partial sums, then fro2 at [kCoopCtas]
};

__host__ __device__ inline size_t big_mat_doubles(int m) {
  const int mp = m + (m & 1);
  return (size_t)mp * (mp + 1);
}

__host__ __device__ inline BigWork big_work(double* w, int m) {
  const size_t mat = big_mat_doubles(m);
  BigWork b;
  b.A32 = reinterpret_cast<float*>(w);
  b.Q32 = reinterpret_cast<float*>(w) + mat;
  b.A = w + mat;
  b.Q = b.A + mat;
  b.W = b.Q + mat;
  b.S = b.W + mat;
  b.bar = reinterpret_cast<unsigned*>(b.S + mat);
  b.part = b.S + mat + 4;
  return b;
}

size_t ritz_work_doubles(int m) {
  const int mp = m + (m & 1);
  if (m <= kRitzSmallMax) return 0;
  if (m <= kRitzMidMax) return (size_t)2 * mp * (mp + 1);
  return 5 * big_mat_doubles(m) + 4 + kCoopCtas + 8;
}

// 1. FP32 sweeps (one CTA) and the FP64 copies of T and Q32.
__global__ void __launch_bounds__(1024) ritz_big_fp32_kernel(const double* __restrict__ H, int m, double* work) {
  const int mp = m + (m & 1), ld = mp + 1, np = mp / 2;
  BigWork w = big_work(work, m);
  __shared__ float cs[kRitzMax / 2], sn[kRitzMax / 2];
  __shared__ int pp[kRitzMax / 2], pq[kRitzMax / 2];
  __shared__ double red[32];
  __shared__ bool conv;
  const int tid = threadIdx.x, nth = blockDim.x;
  double v = 0.0;
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    const double a = (i < m && j < m) ? 0.5 * (H[i * m + j] + H[j * m + i]) : 0.0;
    w.A32[i * ld + j] = (float)a;
    w.Q32[i * ld + j] = (i == j) ? 1.f : 0.f;
    v += a * a;
  }
  const double fro2 = ritz_block_sum(v, red);
  __syncthreads();
  jacobi_sweeps<float>(w.A32, w.Q32, ld, m, mp, 1e-12 * fro2, 20, cs, sn, pp, pq, red, &conv);
  for (int e = tid; e < mp * mp; e += nth) {
    const int i = e / mp, j = e % mp;
    w.Q[i * ld + j] = (double)w.Q32[i * ld + j];
    w.A[i * ld + j] = (i < m && j < m) ? 0.5 * (H[i * m + j] + H[j * m + i]) : 0.0;
  }
  if (tid == 0) w.part[kCoopCtas] = fro2;
  (void)np;
}

// 2. C = alpha op(A) op(B) + beta C for mp x mp FP64 matrices (row stride ld); op = transpose
// when ta / tb.  32 x 32 output tile per CTA, 256 threads with 4 outputs each.
__global__ void __launch_bounds__(256) ritz_dgemm_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                         double* __restrict__ C, int mp, int ld, int ta, int tb,
                                                         double alpha, double beta) {
  __shared__ double sa[32][33], sb[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < mp; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, k = k0 + tx;   // sa[r][tx] = op(A)[i][k]
      sa[r][tx] = (i < mp && k < mp) ? (ta ? A[k * ld + i] : A[i * ld + k]) : 0.0;
      const int kk = k0 + r, j = j0 + tx; // sb[r][tx] = op(B)[kk][j]
      sb[r][tx] = (kk < mp && j < mp) ? (tb ? B[j * ld + kk] : B[kk * ld + j]) : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double bv = sb[k][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(sa[ty + 8 * u][k], bv, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < mp && j < mp) C[i * ld + j] = alpha * acc[u] + (beta != 0.0 ? beta * C[i * ld + j] : 0.0);
  }
}

// Q <- (3 Q - W) / 2 with W = Q (Q^T Q): one Newton-Schulz step.
__global__ void ritz_ns_kernel(double* __restrict__ Q, const double* __restrict__ W, int mp, int ld) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mp * mp) return;
  const int i = e / mp, j = e % mp;
  Q[i * ld + j] = 1.5 * Q[i * ld + j] - 0.5 * W[i * ld + j];
}

// Grid-wide barrier for a cooperative launch (all CTAs resident): arrival counter and
// generation word in global memory.  The wait is bounded; on a timeout the error flag is set
// and false returned (the caller then leaves its loops).
__device__ bool coop_barrier(unsigned* bar, unsigned& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned g = gen;
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      unsigned spins = 0;
      while (atomicAdd(&bar[1], 0u) == g) {
        if (++spins > (1u << 26) || atomicAdd(&bar[2], 0u) != 0u) {
          atomicExch(&bar[2], 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    gen = g + 1;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// 3. FP64 parallel Jacobi sweeps on A (nearly diagonal), Q <- Q J, across the grid.
__global__ void __launch_bounds__(512) ritz_big_jacobi64_kernel(double* work, int m, double tol, int max_sweeps,
                                                                int* info) {
  const int mp = m + (m & 1), ld = mp + 1, np = mp / 2;
  BigWork w = big_work(work, m);
  __shared__ double cs[kRitzMax / 2], sn[kRitzMax / 2];
  __shared__ int pp[kRitzMax / 2], pq[kRitzMax / 2];
  __shared__ double red[32];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int gt = blockIdx.x * nth + tid, gn = gridDim.x * nth;
  unsigned gen = 0;
  const double fro2 = w.part[kCoopCtas];
  const double thresh = tol * tol * fro2;
  int sweeps = 0;
  bool conv = false;
  while (true) {
    double v = 0.0;
    for (int e = gt; e < mp * mp; e += gn) {
      const int i = e / mp, j = e % mp;
      if (i != j) v += w.A[i * ld + j] * w.A[i * ld + j];
    }
    v = ritz_block_sum(v, red);
    if (tid == 0) w.part[blockIdx.x] = v;
    if (!coop_barrier(w.bar, gen)) return;
    double off2 = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) off2 += w.part[c];   // same order in every CTA
    if (off2 <= thresh || sweeps >= max_sweeps) {
      conv = off2 <= thresh;
      break;
    }
    ++sweeps;
    for (int step = 0; step < mp - 1; ++step) {
      // every CTA forms the step's rotations from the same (stable) entries ...
      for (int k = tid; k < np; k += nth) {
        auto pos = [&](int i) { return i == 0 ? 0 : ((i - 1 + step) % (mp - 1)) + 1; };
        int p = pos(k), q = pos(mp - 1 - k);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sv = 0.0;
        if (q < m) {
          const float t = jacobi_tan(w.A[p * ld + p], w.A[p * ld + q], w.A[q * ld + q]);
          if (t != 0.f) jacobi_cs(t, c, sv);
        }
        pp[k] = p;
        pq[k] = q;
        cs[k] = c;
        sn[k] = sv;
      }
      if (!coop_barrier(w.bar, gen)) return;   // all rotations read before any entry changes
      // ... then the CTAs share the independent 2 x 2 block updates and Q's column pairs
      const int nsq = np * np;
      for (int e = gt; e < nsq + mp * np; e += gn) {
        if (e < nsq) {
          const int k = e / np, k2 = e - k * np;
          if (k > k2) continue;
          const double s1 = sn[k], s2 = sn[k2];
          if (s1 == 0.0 && s2 == 0.0) continue;
          const double c1 = cs[k], c2 = cs[k2];
          const int p1 = pp[k], q1 = pq[k];
          double* A = w.A;
          if (k == k2) {
            const double app = A[p1 * ld + p1], aqq = A[q1 * ld + q1], apq = A[p1 * ld + q1];
            const double cc = c1 * c1, ss = s1 * s1, cs2 = c1 * s1;
            A[p1 * ld + p1] = cc * app - 2.0 * cs2 * apq + ss * aqq;
            A[q1 * ld + q1] = ss * app + 2.0 * cs2 * apq + cc * aqq;
            const double npq = cs2 * (app - aqq) + (cc - ss) * apq;
            A[p1 * ld + q1] = npq;
            A[q1 * ld + p1] = npq;
          } else {
            const int p2 = pp[k2], q2 = pq[k2];
            const double x00 = A[p1 * ld + p2], x01 = A[p1 * ld + q2];
            const double x10 = A[q1 * ld + p2], x11 = A[q1 * ld + q2];
            const double y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
            const double y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
            const double z00 = c2 * y00 - s2 * y01, z01 = s2 * y00 + c2 * y01;
            const double z10 = c2 * y10 - s2 * y11, z11 = s2 * y10 + c2 * y11;
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
          const double sk = sn[k];
          if (sk == 0.0) continue;
          const double ck = cs[k];
          const int p = pp[k], q = pq[k];
          const double vp = w.Q[i * ld + p], vq = w.Q[i * ld + q];
          w.Q[i * ld + p] = ck * vp - sk * vq;
          w.Q[i * ld + q] = sk * vp + ck * vq;
        }
      }
      if (!coop_barrier(w.bar, gen)) return;
    }
  }
  if (blockIdx.x == 0 && tid == 0) info[0] = conv ? sweeps : -1;
}

// 4. Ordering and outputs (one CTA).
__global__ void ritz_big_out_kernel(const double* __restrict__ H, int m, int b, int which, double* work,
                                    double* __restrict__ theta_out, double* __restrict__ Y_out,
                                    double* __restrict__ rho_out, int* __restrict__ info) {
  const int mp = m + (m & 1), ld = mp + 1;
  BigWork w = big_work(work, m);
  __shared__ int order[kRitzMax];
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 1; i < m; ++i) {
      const int x = order[i];
      const double tx = w.A[x * ld + x];
      int j = i - 1;
      while (j >= 0) {
        const double ty = w.A[order[j] * ld + order[j]];
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
    if (w.bar[2] != 0u) info[0] = -2;   // a grid barrier timed out
  }
  __syncthreads();
  for (int c = tid; c < m; c += nth) theta_out[c] = w.A[order[c] * ld + order[c]];
  for (int e = tid; e < m * m; e += nth) {
    const int i = e / m, c = e % m;
    Y_out[e] = w.Q[i * ld + order[c]];
  }
  for (int c = tid; c < m; c += nth) {
    double r2 = 0.0;
    for (int p = 0; p < b; ++p) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += H[(m + p) * m + i] * w.Q[i * ld + order[c]];
      r2 += s * s;
    }
    rho_out[c] = sqrt(r2);
  }
}

static int launch_ritz_big(const double* H, int m, int b, int which, int max_sweeps, double tol,
                           double* theta, double* Y, double* rho, int* info, double* work,
                           cudaStream_t s) {
  const int mp = m + (m & 1), ld = mp + 1;
  BigWork w = big_work(work, m);
  FE_CUDA(cudaMemsetAsync(w.bar, 0, 4 * sizeof(unsigned), s));
  ritz_big_fp32_kernel<<<1, 1024, 0, s>>>(H, m, work);
  count_launch();
  FE_CUDA(cudaGetLastError());
  const dim3 gg((mp + 31) / 32, (mp + 31) / 32);
  auto gemm = [&](const double* A, const double* B, double* C, int ta, int tb) -> int {
    ritz_dgemm_kernel<<<gg, 256, 0, s>>>(A, B, C, mp, ld, ta, tb, 1.0, 0.0);
    count_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
  };
  for (int it = 0; it < 2; ++it) {   // Q <- Q (3 I - Q^T Q) / 2
    FE_TRY(gemm(w.Q, w.Q, w.S, 1, 0));
    FE_TRY(gemm(w.Q, w.S, w.W, 0, 0));
    ritz_ns_kernel<<<(mp * mp + 255) / 256, 256, 0, s>>>(w.Q, w.W, mp, ld);
    count_launch();
    FE_CUDA(cudaGetLastError());
  }
  FE_TRY(gemm(w.A, w.Q, w.W, 0, 0));   // W = T Q
  FE_TRY(gemm(w.Q, w.W, w.A, 1, 0));   // A = Q^T T Q
  // cooperative launch: every CTA resident (the grid barrier relies on it)
  static KernelSetup ks;
  int per_sm = 0;
  FE_TRY(kernel_occupancy(ks, reinterpret_cast<const void*>(ritz_big_jacobi64_kernel), 512, 0, 0, &per_sm));
  const int grid = std::min(kCoopCtas, per_sm * num_sms());
  FE_ARG(grid >= 1, "ritz: no resident CTA for the cooperative Jacobi kernel");
  double* wk = work;
  int mm = m, ms = max_sweeps;
  double tl = tol;
  void* args[] = {&wk, &mm, &tl, &ms, &info};
  FE_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(ritz_big_jacobi64_kernel), dim3(grid),
                                      dim3(512), args, 0, s));
  count_launch();
  ritz_big_out_kernel<<<1, 512, 0, s>>>(H, m, b, which, work, theta, Y, rho, info);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int launch_ritz(const double* H, int m, int b, int which, int max_sweeps, double tol,
                double* theta, double* Y, double* rho, int* info, double* work, cudaStream_t s) {
  FE_ARG(m >= 1 && m <= kRitzMax, "ritz: subspace m = %d not in [1, %d]", m, kRitzMax);
  if (m > kRitzMidMax) {
    FE_ARG(work != nullptr, "ritz: m = %d needs a global workspace", m);
    return launch_ritz_big(H, m, b, which, max_sweeps, tol, theta, Y, rho, info, work, s);
  }
  const size_t smem = ritz_smem_bytes(m);
  FE_ARG(smem <= 225 * 1024, "ritz: subspace m = %d too large", m);
  const bool big = m > kRitzSmallMax;
  FE_ARG(!big || work != nullptr, "ritz: m = %d needs a global workspace", m);
  static KernelSetup ks[2];
  FE_TRY(kernel_configure(ks[big], big ? reinterpret_cast<const void*>(ritz_kernel<true>)
                                       : reinterpret_cast<const void*>(ritz_kernel<false>),
                          225 * 1024));
  // one CTA: a rotation step is (m/2)^2 / 2 2 x 2 blocks plus m^2 / 2 Q updates between two
  // barriers; FP64 work on one SM runs at 2 DFMA per clock, hence the FP32 sweeps first, and
  // 1024 threads, so that many independent FP64 chains hide the FP64 pipe's latency
  if (big)
    ritz_kernel<true><<<1, 1024, smem, s>>>(H, m, b, which, max_sweeps, tol, theta, Y, rho, info, work);
  else
    ritz_kernel<false><<<1, 1024, smem, s>>>(H, m, b, which, max_sweeps, tol, theta, Y, rho, info, nullptr);
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
