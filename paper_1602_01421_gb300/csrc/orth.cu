// Re-orthogonalisation of a new Krylov block (Section 3.1 step (1); the paper notes that
// MvTransMv and MvTimesMatAddMv are spent mainly here, Section 3.4).
//
// W_in = V G + W_out R with W_out orthonormal and orthogonal to V:
//   pass 1  [G1; S1] = [V W]^T W        (Gram, one sweep; S1 = W^T W gives the ||A|| estimate)
//           W <- W - V G1
//   pass 2  [G2; S] = [V W]^T W         (Gram; S - G2^T G2 = W^T W after the next update)
//           R1 = chol(S - G2^T G2)      (CholeskyQR pass 1, pivots checked)
//           W <- (W - V G2) R1^{-1}     (one fused update)
//   pass 3  R2 = chol(W^T W),  W <- W R2^{-1},  R = R2 R1   (CholeskyQR pass 2)
// With pass1_f32 (the solver's default for FP64 subspaces) the pass-1 Gram runs in FP32
// arithmetic -- G1 only steers the subtraction, and H records G1 + G2, what was subtracted --
// and pass 2's correction V C (C = -G2 R1^{-1}, entries below 1e-5) is formed in FP32
// arithmetic and added to the FP64 W R1^{-1}; all other products are FP64.
// The small b x b / k x b algebra runs in single-CTA kernels; updates after a failed pivot
// check are skipped on the device and the host finishes with column-wise two-pass
// Gram-Schmidt, replacing a column whose remainder is below 1e-12 ||A|| by a random
// direction (breakdown of the Krylov space).  One host synchronisation per call.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fe_internal.cuh"
#include "vec.cuh"

namespace fe {

int update_skip(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                const double* M, void* W, int bw, int ldw, fe_dtype dt, const int* skip,
                cudaStream_t s);
int gram_f32_arith(const BlockSet& V, int64_t n, const double* W, int b, double alpha, double* G,
                   cudaStream_t s);
int update_tri_gram(const BlockSet& V, int64_t n, const double* C, double alpha, double beta,
                    const double* M, void* W, int b, fe_dtype dt, const int* skip, const int* vc32,
                    double* S, cudaStream_t s);

constexpr double kRelPivot = 1e-6;      // pivot below 1e-6 * column norm: nearly dependent
constexpr double kAbsBreakdown = 1e-12; // remainder below 1e-12 * ||A||: breakdown
// Second-pass correction coefficients C = -G2 R1^{-1} at most this large (W's columns have unit
// scale after R1^{-1}) are applied in FP32 arithmetic: the FP32 rounding of V C is then below
// 2^-23 * 1e-5 * (sum_j |V_j[r]|), under 1e-12 of W even in the worst case and ~1e-15 typically.
constexpr double kSmallCorrection = 1e-5;

// Upper-triangular R (row-major b x b) with R^T R = S; false if a pivot check fails.
__device__ bool chol_upper_dev(const double* S, int b, double rel, double absthr, double* R) {
  for (int e = 0; e < b * b; ++e) R[e] = 0.0;
  for (int j = 0; j < b; ++j) {
    for (int i = 0; i < j; ++i) {
      double s = S[i * b + j];
      for (int l = 0; l < i; ++l) s -= R[l * b + i] * R[l * b + j];
      R[i * b + j] = s / R[i * b + i];
    }
    double d = S[j * b + j];
    for (int l = 0; l < j; ++l) d -= R[l * b + j] * R[l * b + j];
    if (!(d > 0.0)) return false;
    const double rd = sqrt(d);
    if (rd < rel * sqrt(fmax(S[j * b + j], 0.0)) || rd <= absthr) return false;
    R[j * b + j] = rd;
  }
  return true;
}

// Ri = R^{-1} for upper-triangular R (back substitution, column by column).
__device__ void inv_upper_dev(const double* R, int b, double* Ri) {
  for (int e = 0; e < b * b; ++e) Ri[e] = 0.0;
  for (int c = 0; c < b; ++c) {
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) s -= R[i * b + l] * Ri[l * b + c];
      Ri[i * b + c] = s / R[i * b + i];
    }
  }
}

// After pass 2.  G1x = [G1; S1] ((k+b) x b), G2x = [G2; S] ((k+b) x b); k may be 0 (then
// G2x = S).  Writes G (k x b, ldg), Racc = R1, M = R1^{-1}, C = -G2 R1^{-1}; on a failed check
// sets *status = 1, G = G1, Racc = I.  status[1] = 1 when max |C| <= kSmallCorrection.
__global__ void orth_post2_kernel(const double* __restrict__ G1x, const double* __restrict__ G2x,
                                  int k, int b, double* __restrict__ anorm, int update_anorm,
                                  double* __restrict__ G, int ldg, double* __restrict__ Racc,
                                  double* __restrict__ M, double* __restrict__ C,
                                  int* __restrict__ status) {
  __shared__ double S[256], R[256], Ri[256];
  __shared__ int ok;
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e % b;
    double s = G2x[(k + p) * b + q];
    for (int i = 0; i < k; ++i) s -= G2x[i * b + p] * G2x[i * b + q];
    S[e] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double a = *anorm;
    if (update_anorm) {
      for (int p = 0; p < b; ++p) a = fmax(a, sqrt(fmax(G1x[(k + p) * b + p], 0.0)));
      *anorm = a;
    }
    ok = chol_upper_dev(S, b, kRelPivot, kAbsBreakdown * a, R) ? 1 : 0;
    if (ok) inv_upper_dev(R, b, Ri);
    else *status = 1;
  }
  __syncthreads();
  for (int e = tid; e < k * b; e += blockDim.x) {
    const int i = e / b, q = e % b;
    if (ok) {
      G[i * ldg + q] = G1x[i * b + q] + G2x[i * b + q];
      double c = 0.0;
      for (int p = 0; p <= q; ++p) c -= G2x[i * b + p] * Ri[p * b + q];
      C[e] = c;
    } else {
      G[i * ldg + q] = G1x[i * b + q];
    }
  }
  for (int e = tid; e < b * b; e += blockDim.x) {
    if (ok) {
      Racc[e] = R[e];
      M[e] = Ri[e];
    } else {
      Racc[e] = (e / b == e % b) ? 1.0 : 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double cmax = 0.0;
    if (ok)
      for (int e = 0; e < k * b; ++e) cmax = fmax(cmax, fabs(C[e]));
    status[1] = (ok && cmax <= kSmallCorrection) ? 1 : 0;
  }
}

// After pass 3: R2 = chol(S2); R = R2 Racc (-> Rout, ldr), M = R2^{-1}; failure -> *status = 2.
__global__ void orth_post3_kernel(const double* __restrict__ S2, int b,
                                  const double* __restrict__ Racc, double* __restrict__ M,
                                  double* __restrict__ Rout, int ldr, int* __restrict__ status) {
  __shared__ double R2[256], Ri[256];
  __shared__ int ok;
  if (*status) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    ok = chol_upper_dev(S2, b, kRelPivot, 0.0, R2) ? 1 : 0;
    if (ok) inv_upper_dev(R2, b, Ri);
    else *status = 2;
  }
  __syncthreads();
  if (!ok) return;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e % b;
    double r = 0.0;
    for (int l = p; l <= q; ++l) r += R2[p * b + l] * Racc[l * b + q];
    Rout[p * ldr + q] = r;
    M[e] = Ri[e];
  }
  if (tid == 0) {  // status[2]: R2^{-1} is the identity up to kSmallCorrection
    double dmax = 0.0;
    for (int e = 0; e < b * b; ++e) dmax = fmax(dmax, fabs(Ri[e] - (e / b == e % b ? 1.0 : 0.0)));
    status[2] = dmax <= kSmallCorrection ? 1 : 0;
  }
}

// W <- W M for the second CholeskyQR pass (M = R2^{-1}), skipped after a failed check.  After
// an FP64 first pass M is the identity to about 1e-15; when allow32 and status[2] say every
// |M - I| entry is at most kSmallCorrection, the product is taken as W + W (M - I) with the
// correction in FP32 arithmetic (W converted by integer truncation), far below FP64 rounding of W.
template <typename T, int B>
__global__ void __launch_bounds__(256) right_mult_kernel(T* __restrict__ W, int64_t n,
                                                         const double* __restrict__ M,
                                                         const int* __restrict__ status, int allow32) {
  if (status[0]) return;
  __shared__ T sM[B * B];
  __shared__ float sD[B * B];
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    sM[e] = (T)M[e];
    sD[e] = (float)(M[e] - (e / B == e % B ? 1.0 : 0.0));
  }
  __syncthreads();
  const bool small = sizeof(T) == 8 && allow32 && status[2] != 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    T w[B], out[B];
    ld_row_rw<T, B>(W + r * B, w);
    if (small) {
      float wf[B];
#pragma unroll
      for (int p = 0; p < B; ++p) wf[p] = f64_to_f32_trunc((double)w[p]);
#pragma unroll
      for (int q = 0; q < B; ++q) {
        float c = 0.f;
#pragma unroll
        for (int p = 0; p < B; ++p) c = fmaf(wf[p], sD[p * B + q], c);
        out[q] = w[q] + (T)f32_to_f64_flush(c);
      }
    } else {
#pragma unroll
      for (int q = 0; q < B; ++q) {
        T x = T(0);
#pragma unroll
        for (int p = 0; p < B; ++p) x = fma(w[p], sM[p * B + q], x);
        out[q] = x;
      }
    }
    st_row<T, B>(W + r * B, out);
  }
}

template <typename T>
static int launch_right_mult(T* W, int64_t n, int b, const double* M, const int* status,
                             int allow32, cudaStream_t s) {
  const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * num_sms()));
  switch (b) {
    case 1: right_mult_kernel<T, 1><<<ctas, 256, 0, s>>>(W, n, M, status, allow32); break;
    case 2: right_mult_kernel<T, 2><<<ctas, 256, 0, s>>>(W, n, M, status, allow32); break;
    case 4: right_mult_kernel<T, 4><<<ctas, 256, 0, s>>>(W, n, M, status, allow32); break;
    case 8: right_mult_kernel<T, 8><<<ctas, 256, 0, s>>>(W, n, M, status, allow32); break;
    case 16: right_mult_kernel<T, 16><<<ctas, 256, 0, s>>>(W, n, M, status, allow32); break;
    default: return set_error(FE_ERR_INVALID, "orth: b = %d", b);
  }
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

__global__ void add_col_kernel(double* __restrict__ dst, int ld, int col,
                               const double* __restrict__ src, int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i * ld + col] += src[i];
}

__global__ void set_value_kernel(double* dst, double v) { *dst = v; }

// G = Gacc + Gf Racc (k x b, G with ldg); R = Rf Racc (b x b, ldr).
__global__ void compose_kernel(double* __restrict__ G, int ldg, const double* __restrict__ Gf,
                               const double* __restrict__ Racc, const double* __restrict__ Rf,
                               double* __restrict__ R, int ldr, int k, int b) {
  for (int e = threadIdx.x; e < k * b; e += blockDim.x) {
    const int i = e / b, q = e % b;
    double s = 0.0;
    for (int l = 0; l < b; ++l) s += Gf[i * b + l] * Racc[l * b + q];
    G[i * ldg + q] += s;
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e % b;
    double s = 0.0;
    for (int l = 0; l < b; ++l) s += Rf[p * b + l] * Racc[l * b + q];
    R[p * ldr + q] = s;
  }
}

static int read_scalar(const double* d, double* h, cudaStream_t s) {
  FE_CUDA(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaStreamSynchronize(s));
  return FE_OK;
}

static int col_norm(void* wi, int64_t n, int ld, fe_dtype dt, double* tmp, double* out,
                    cudaStream_t s) {
  BlockSet one = blockset_of({wi}, 1, ld);
  FE_TRY(gram(one, n, wi, 1, ld, dt, 1.0, tmp, s));
  double v = 0.0;
  FE_TRY(read_scalar(tmp, &v, s));
  *out = sqrt(fmax(v, 0.0));
  return FE_OK;
}

// Column-wise two-pass Gram-Schmidt with random replacement, continuing from
// W_in = V Gacc + W Racc (Gacc in G with ldg, Racc device b x b).
static int orth_fallback(const BlockSet& V, int64_t n, void* W, int b, fe_dtype dt,
                         double anorm, uint64_t seed, uint64_t* counter, double* G, int ldg,
                         const double* Racc, double* Rout, int ldr, int* replaced,
                         cudaStream_t s) {
  const int k = V.nv * b;
  const size_t es = dt_size(dt);
  double* Gf = small_scratch(8, (size_t)std::max(k, 1) * b);
  double* Rf = small_scratch(9, (size_t)b * b);
  double* tmp = small_scratch(10, (size_t)k + b + 1);
  if (!Gf || !Rf || !tmp) return FE_ERR_OOM;
  FE_CUDA(cudaMemsetAsync(Gf, 0, sizeof(double) * std::max(k, 1) * b, s));
  FE_CUDA(cudaMemsetAsync(Rf, 0, sizeof(double) * b * b, s));
  for (int i = 0; i < b; ++i) {
    void* wi = (char*)W + (size_t)i * es;
    std::vector<const void*> qcols;
    for (int c = 0; c < i; ++c) qcols.push_back((const char*)W + (size_t)c * es);
    BlockSet Q = blockset_of(qcols, 1, b);
    auto project = [&](bool record) -> int {
      for (int pass = 0; pass < 2; ++pass) {
        if (V.nv > 0) {
          FE_TRY(gram(V, n, wi, 1, b, dt, 1.0, tmp, s));
          FE_TRY(update(V, n, tmp, -1.0, 1.0, nullptr, wi, 1, b, dt, s));
          if (record) { add_col_kernel<<<1, 256, 0, s>>>(Gf, b, i, tmp, k); count_launch(); }
        }
        if (i > 0) {
          FE_TRY(gram(Q, n, wi, 1, b, dt, 1.0, tmp, s));
          FE_TRY(update(Q, n, tmp, -1.0, 1.0, nullptr, wi, 1, b, dt, s));
          if (record) { add_col_kernel<<<1, 256, 0, s>>>(Rf, b, i, tmp, i); count_launch(); }
        }
        FE_CUDA(cudaGetLastError());
      }
      return FE_OK;
    };
    FE_TRY(project(true));
    double nr = 0.0;
    FE_TRY(col_norm(wi, n, b, dt, tmp, &nr, s));
    if (nr > kAbsBreakdown * anorm && nr > 0.0) {
      BlockSet none = blockset_of({}, 1, b);
      FE_TRY(update(none, n, nullptr, 0.0, 1.0 / nr, nullptr, wi, 1, b, dt, s));
      set_value_kernel<<<1, 1, 0, s>>>(Rf + i * b + i, nr);
      count_launch();
      FE_CUDA(cudaGetLastError());
      continue;
    }
    bool ok = false;
    for (int attempt = 0; attempt < 8 && !ok; ++attempt) {
      FE_TRY(random_normal(wi, n, 1, b, dt, seed, 5, (*counter) * (uint64_t)n, s));
      *counter += 1;
      double r0 = 0.0;
      FE_TRY(col_norm(wi, n, b, dt, tmp, &r0, s));
      FE_TRY(project(false));
      FE_TRY(col_norm(wi, n, b, dt, tmp, &nr, s));
      if (nr > 1e-10 * r0) {
        BlockSet none = blockset_of({}, 1, b);
        FE_TRY(update(none, n, nullptr, 0.0, 1.0 / nr, nullptr, wi, 1, b, dt, s));
        ok = true;
      }
    }
    if (!ok) return set_error(FE_ERR_INVALID, "orth: cannot find a replacement direction (subspace fills R^n)");
    if (replaced) *replaced += 1;
  }
  compose_kernel<<<1, 256, 0, s>>>(G, ldg, Gf, Racc, Rf, Rout, ldr, k, b);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// sG1 ((k + b) x b, rows j*b + p for block j's column p, then the b rows of S1): rows of the
// older blocks from the known coefficients (row r, column q = known[q * ldk + r], blocks below
// nz_first zero), the newest block's rows and S1 from the local Gram [v_last W]^T W (2b x b).
__global__ void known_g1_kernel(double* __restrict__ sG1, int k, int b, const double* __restrict__ known,
                                int ldk, int nz_first, const double* __restrict__ local) {
  const int kold = k - b;
  for (int e = threadIdx.x; e < (k + b) * b; e += blockDim.x) {
    const int r = e / b, q = e - (e / b) * b;
    double x;
    if (r < kold) x = r / b >= nz_first ? known[(size_t)q * ldk + r] : 0.0;
    else x = local[(r - kold) * b + q];
    sG1[e] = x;
  }
}

int orth_ex(const BlockSet& V, int64_t n, void* W, int b, fe_dtype dt, double* d_anorm,
            int update_anorm, uint64_t seed, uint64_t* rng_counter, double* d_G, int ldg,
            double* d_R, int ldr, int* replaced, cudaStream_t s, int pass1_f32, int engine,
            const double* d_known, int ldk, int nz_first) {
  FE_ARG(V.nv >= 0 && V.nv + 1 <= kMaxBlocks, "orth: too many blocks");
  FE_ARG(b >= 1 && b <= 16, "orth: b = %d", b);
  const int k = V.nv * b;
  double* sG1 = small_scratch(1, (size_t)(k + b) * b);
  double* sG2 = small_scratch(2, (size_t)(k + b) * b);
  double* sM = small_scratch(3, (size_t)b * b);
  double* sC = small_scratch(4, (size_t)std::max(k, 1) * b);
  double* sRacc = small_scratch(5, (size_t)b * b);
  double* sS2 = small_scratch(6, (size_t)b * b);
  double* sStat = small_scratch(7, 2);
  double* gdummy = small_scratch(11, (size_t)b);
  if (!sG1 || !sG2 || !sM || !sC || !sRacc || !sS2 || !sStat || !gdummy) return FE_ERR_OOM;
  int* status = reinterpret_cast<int*>(sStat);
  if (!d_G) d_G = gdummy;  // k == 0: nothing is written to G
  FE_CUDA(cudaMemsetAsync(status, 0, 3 * sizeof(int), s));
  std::vector<const void*> vx(V.blk, V.blk + V.nv);
  vx.push_back(W);
  BlockSet Vx = blockset_of(vx, b, b);
  FE_ARG(V.nv == 0 || V.bv == b, "orth: V block width %d != b %d", V.bv, b);
  // pass 1: [G1; S1] = [V W]^T W (FP64 blocks: optionally in FP32 arithmetic -- G1 only steers
  // the first subtraction; pass 2 is FP64, and H receives G1 + G2, what was actually subtracted).
  // With known coefficients (d_known: the solver's symmetric projected matrix) only the newest
  // block's rows and S1 are computed, [v_last W]^T W; the first update then involves blocks
  // nz_first .. last only.
  const bool local = d_known != nullptr && V.nv > 0;
  int v0 = 0;   // first block of the first update
  if (local) {
    FE_ARG(nz_first >= 0 && nz_first < V.nv, "orth: nz_first = %d", nz_first);
    v0 = nz_first;
    BlockSet Vl = blockset_of({V.blk[V.nv - 1], W}, b, b);
    double* sLoc = small_scratch(19, (size_t)2 * b * b);
    if (!sLoc) return FE_ERR_OOM;
    if (pass1_f32 && dt == FE_F64)
      FE_TRY(gram_f32_arith(Vl, n, static_cast<const double*>(W), b, 1.0, sLoc, s));
    else
      FE_TRY(gram(Vl, n, W, b, b, dt, 1.0, sLoc, s));
    known_g1_kernel<<<1, 256, 0, s>>>(sG1, k, b, d_known, ldk, nz_first, sLoc);
    count_launch();
    FE_CUDA(cudaGetLastError());
  } else if (pass1_f32 && dt == FE_F64) {
    FE_TRY(gram_f32_arith(Vx, n, static_cast<const double*>(W), b, 1.0, sG1, s));
  } else {
    FE_TRY(gram(Vx, n, W, b, b, dt, 1.0, sG1, s));
  }
  // the fused update + Gram sweeps hold a b x b accumulator per lane: b = 16 keeps two kernels
  const bool fused = b <= 8;
  // FP64 blocks on the tensor cores (engine AUTO or TC): the update as a split-product block
  // product with the FP64 W added, the Gram as split products with per-tile column scaling
  // (scale 22, b = 4: 6.54 s against 6.67 s per solve with the fused FMA sweep)
  BlockSet Wset = blockset_of({W}, b, b);
  const bool tc2 = V.nv > 0 && engine != FE_ENGINE_FMA && dt == FE_F64 &&
                   tc_combine_supported(V, Wset, dt) && tc_gram_supported(Vx, b, b, dt);
  if (tc2) {
    std::vector<const void*> vu(V.blk + v0, V.blk + V.nv);
    BlockSet Vu = blockset_of(vu, b, b);
    FE_TRY(tc_combine(Vu, n, sG1 + (size_t)v0 * b * b, b, Wset, s, -1.0, 1.0));   // W <- W - V G1
    FE_TRY(tc_gram(Vx, n, static_cast<const double*>(W), b, 1.0, sG2, s));  // [G2; S]
    orth_post2_kernel<<<1, 256, 0, s>>>(sG1, sG2, k, b, d_anorm, update_anorm, d_G, ldg, sRacc,
                                        sM, sC, status);
  } else if (V.nv > 0) {
    // W <- W - V G1 and [G2; S] = [V W]^T W in one sweep
    if (fused) {
      FE_TRY(update_gram(V, n, sG1, -1.0, 1.0, nullptr, W, b, dt, 1, nullptr, sG2, s));
    } else {
      FE_TRY(update(V, n, sG1, -1.0, 1.0, nullptr, W, b, b, dt, s));
      FE_TRY(gram(Vx, n, W, b, b, dt, 1.0, sG2, s));
    }
    orth_post2_kernel<<<1, 256, 0, s>>>(sG1, sG2, k, b, d_anorm, update_anorm, d_G, ldg, sRacc,
                                        sM, sC, status);
  } else {
    orth_post2_kernel<<<1, 256, 0, s>>>(sG1, sG1, 0, b, d_anorm, update_anorm, d_G, ldg, sRacc,
                                        sM, sC, status);
  }
  count_launch();
  FE_CUDA(cudaGetLastError());
  // W <- (W - V G2) R1^{-1} and S2 = W^T W in one sweep (skipped after a failed pivot check)
  if (fused && b <= 4) {
    // M = R1^{-1} is upper triangular: thread-per-row sweep over its triangle, S2 = W^T W in
    // per-thread accumulators; for FP64 blocks the correction V C in FP32 arithmetic when it
    // is tiny
    FE_TRY(update_tri_gram(V, n, sC, 1.0, 1.0, sM, W, b, dt, status,
                           (pass1_f32 && dt == FE_F64) ? status + 1 : nullptr, sS2, s));
  } else if (fused) {
    // the correction V C in FP32 arithmetic when it is tiny (FP64 subspace, pass1_f32 mode)
    FE_TRY(update_gram(V, n, sC, 1.0, 1.0, sM, W, b, dt, 0, status, sS2, s,
                       (pass1_f32 && dt == FE_F64) ? status + 1 : nullptr));
  } else {
    FE_TRY(update_skip(V, n, sC, 1.0, 1.0, sM, W, b, b, dt, status, s));
    BlockSet Wonly = blockset_of({W}, b, b);
    FE_TRY(gram(Wonly, n, W, b, b, dt, 1.0, sS2, s));
  }
  orth_post3_kernel<<<1, 64, 0, s>>>(sS2, b, sRacc, sM, d_R, ldr, status);
  count_launch();
  FE_CUDA(cudaGetLastError());
  const int allow32 = (pass1_f32 && dt == FE_F64) ? 1 : 0;
  if (dt == FE_F64) FE_TRY(launch_right_mult(static_cast<double*>(W), n, b, sM, status, allow32, s));
  else FE_TRY(launch_right_mult(static_cast<float*>(W), n, b, sM, status, 0, s));
  int st = 0;
  double an = 0.0;
  FE_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaMemcpyAsync(&an, d_anorm, sizeof(double), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaStreamSynchronize(s));
  if (st == 0) return FE_OK;
  return orth_fallback(V, n, W, b, dt, an, seed, rng_counter, d_G, ldg, sRacc, d_R, ldr,
                       replaced, s);
}

int orth(const BlockSet& V, int64_t n, void* W, int b, fe_dtype dt, double* d_anorm,
         double anorm_floor, uint64_t seed, uint64_t* rng_counter, double* d_G, int ldg,
         double* d_R, int ldr, int* replaced, cudaStream_t s) {
  (void)anorm_floor;
  return orth_ex(V, n, W, b, dt, d_anorm, 0, seed, rng_counter, d_G, ldg, d_R, ldr, replaced, s, 0,
                 FE_ENGINE_FMA, nullptr, 0, 0);
}

}  // namespace fe
