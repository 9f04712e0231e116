// Learned start block (not in the paper; an extension of its random start, Table 1 MvRandom):
// features from SpMM powers (Section 3.3's operation), a 3-layer MLP that maps them to an
// n x b block, its training kernels (loss, gradient, Adam), and the start block fe_eigs uses.
//
// Features (8 per vertex; rms(x) = sqrt(mean(x^2)), 1 when 0):
//   d = A 1; f0 = log(1+d), f1 = d/rms(d), f2 = A d/rms, f3 = A^2 d/rms;
//   R = N(0,1) n x 4 (counter RNG, stream 6); q_p = mean_c (A^p R)_{:,c}^2 (p = 2, 3, 4);
//   f4 = q2/rms(q2), f5 = q3/rms(q3), f6 = q4/rms(q4), f7 = log(1 + q2/mean(q2)).
// Network: h1 = relu(F W1 + b1), h2 = relu(h1 W2 + b2), Z = h2 W3 + b3; parameters packed
// [W1 (8 x H), b1, W2 (H x H), b2, W3 (H x b), b3], FP32.
// Loss against unit reference columns U: L = sum_j (1 - (z_j . u_j)^2 / |z_j|^2).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

constexpr int kNFeat = 8;
constexpr uint64_t kStreamProbe = 6;

int64_t mlp_param_count(int H, int b) {
  return (int64_t)kNFeat * H + H + (int64_t)H * H + H + (int64_t)H * b + b;
}

// ---------------------------------------------------------------- features
__global__ void fill_kernel(double* x, int64_t n, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

// q[i] = mean over the 4 columns of P[i][c]^2
__global__ void rowmeansq_kernel(const double* __restrict__ P, int64_t n, double* __restrict__ q) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = P[4 * i], b = P[4 * i + 1], c = P[4 * i + 2], d = P[4 * i + 3];
    q[i] = 0.25 * (a * a + b * b + c * c + d * d);
  }
}

// sums[k] = sum_i x_k[i]^2 for the 6 vectors, sums[6] = sum_i q2[i]; per-CTA partials.
struct FeatVecs {
  const double* v[6];
  const double* q2;
};
__global__ void feat_sums_kernel(const FeatVecs fv, int64_t n, double* __restrict__ partial) {
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double x = fv.v[k][i];
      acc[k] += x * x;
    }
    acc[6] += fv.q2[i];
  }
  __shared__ double red[7][256];
#pragma unroll
  for (int k = 0; k < 7; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 7; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 7) partial[blockIdx.x * 7 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void feat_scales_kernel(const double* __restrict__ partial, int nctas, int64_t n,
                                   double* __restrict__ scale) {
  const int k = threadIdx.x;
  if (k >= 7) return;
  double s = 0.0;
  for (int c = 0; c < nctas; ++c) s += partial[c * 7 + k];
  const double m = s / (double)n;
  if (k < 6) {
    const double r = sqrt(m);
    scale[k] = r > 0.0 ? r : 1.0;   // rms
  } else {
    scale[k] = m > 0.0 ? m : 1.0;   // mean(q2)
  }
}

__global__ void feat_assemble_kernel(const FeatVecs fv, int64_t n, const double* __restrict__ scale,
                                     float* __restrict__ F) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = fv.v[0][i];
    float* f = F + i * kNFeat;
    f[0] = (float)log1p(d);
    f[1] = (float)(d / scale[0]);
    f[2] = (float)(fv.v[1][i] / scale[1]);
    f[3] = (float)(fv.v[2][i] / scale[2]);
    f[4] = (float)(fv.v[3][i] / scale[3]);
    f[5] = (float)(fv.v[4][i] / scale[4]);
    f[6] = (float)(fv.v[5][i] / scale[5]);
    f[7] = (float)log1p(fv.q2[i] / scale[6]);
  }
}

static int spmm_any(fe_csr h, const void* X, void* Y, int b, cudaStream_t s) {
  if (h->semi_external) return semiext_spmm(h, X, Y, b, FE_F64, s);
  return spmm_resident(h, X, Y, b, FE_F64, s);
}

int vertex_features(fe_csr h, uint64_t seed, float* F, cudaStream_t s) {
  const int64_t n = h->n;
  DevBuf buf;
  // d, ad, a2d, q2, q3, q4 (n each) + R/P ping-pong (2 x 4n)
  FE_TRY(buf.alloc(sizeof(double) * (size_t)n * 14));
  double* d = buf.as<double>();
  double* ad = d + n;
  double* a2d = ad + n;
  double* q2 = a2d + n;
  double* q3 = q2 + n;
  double* q4 = q3 + n;
  double* P0 = q4 + n;
  double* P1 = P0 + 4 * n;
  double* ones = P1;  // scratch before the probes use it
  const int ctas = (int)std::min<int64_t>(ceil_div(n, 256), 4 * num_sms());
  fill_kernel<<<ctas, 256, 0, s>>>(ones, n, 1.0);
  count_launch();
  FE_CUDA(cudaGetLastError());
  FE_TRY(spmm_any(h, ones, d, 1, s));
  FE_TRY(spmm_any(h, d, ad, 1, s));
  FE_TRY(spmm_any(h, ad, a2d, 1, s));
  FE_TRY(random_normal(P0, n, 4, 4, FE_F64, seed, kStreamProbe, 0, s));
  FE_TRY(spmm_any(h, P0, P1, 4, s));   // A R
  FE_TRY(spmm_any(h, P1, P0, 4, s));   // A^2 R
  rowmeansq_kernel<<<ctas, 256, 0, s>>>(P0, n, q2);
  count_launch();
  FE_TRY(spmm_any(h, P0, P1, 4, s));   // A^3 R
  rowmeansq_kernel<<<ctas, 256, 0, s>>>(P1, n, q3);
  count_launch();
  FE_TRY(spmm_any(h, P1, P0, 4, s));   // A^4 R
  rowmeansq_kernel<<<ctas, 256, 0, s>>>(P0, n, q4);
  count_launch();
  FE_CUDA(cudaGetLastError());
  FeatVecs fv;
  fv.v[0] = d;
  fv.v[1] = ad;
  fv.v[2] = a2d;
  fv.v[3] = q2;
  fv.v[4] = q3;
  fv.v[5] = q4;
  fv.q2 = q2;
  const int rctas = (int)std::min<int64_t>(ceil_div(n, 256), 2 * num_sms());
  double* part = small_scratch(14, (size_t)rctas * 7 + 8);
  if (!part) return FE_ERR_OOM;
  double* scale = part + (size_t)rctas * 7;
  feat_sums_kernel<<<rctas, 256, 0, s>>>(fv, n, part);
  count_launch();
  feat_scales_kernel<<<1, 32, 0, s>>>(part, rctas, n, scale);
  count_launch();
  feat_assemble_kernel<<<ctas, 256, 0, s>>>(fv, n, scale, F);
  count_launch();
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaStreamSynchronize(s));  // buf is freed on return
  return FE_OK;
}

// ---------------------------------------------------------------- forward
template <int H, int B>
struct MlpParams {
  static constexpr int W1 = 0, B1 = kNFeat * H, W2 = B1 + H, B2 = W2 + H * H, W3 = B2 + H,
                       B3 = W3 + H * B, COUNT = B3 + B;
};

// One row through the network.  h1 stays in registers; each h2 unit is folded into z as soon
// as it is computed (and optionally stored to h2_out), so no h2 array is kept.
template <int H, int B>
__device__ __forceinline__ void mlp_row_forward(const float* __restrict__ sp, const float* f,
                                                float* h1, float* z, float* h2_out) {
  using P = MlpParams<H, B>;
#pragma unroll
  for (int q = 0; q < H; ++q) {
    float a = sp[P::B1 + q];
#pragma unroll
    for (int i = 0; i < kNFeat; ++i) a = fmaf(f[i], sp[P::W1 + i * H + q], a);
    h1[q] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int j = 0; j < B; ++j) z[j] = sp[P::B3 + j];
#pragma unroll 1
  for (int q = 0; q < H; ++q) {
    float a = sp[P::B2 + q];
#pragma unroll
    for (int p = 0; p < H; ++p) a = fmaf(h1[p], sp[P::W2 + p * H + q], a);
    const float h2q = fmaxf(a, 0.0f);
    if (h2_out) h2_out[q] = h2q;
#pragma unroll
    for (int j = 0; j < B; ++j) z[j] = fmaf(h2q, sp[P::W3 + q * B + j], z[j]);
  }
}

template <int H, int B>
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ F, int64_t n,
                                                          const float* __restrict__ params,
                                                          float* __restrict__ Z) {
  using P = MlpParams<H, B>;
  __shared__ float sp[P::COUNT];
  for (int e = threadIdx.x; e < P::COUNT; e += blockDim.x) sp[e] = params[e];
  __syncthreads();
#pragma unroll 1
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // keep the weight loads inside the loop (hoisting 64 x 64 shared loads spills registers)
    asm volatile("" ::: "memory");
    float f[kNFeat], h1[H], z[B];
#pragma unroll
    for (int k = 0; k < kNFeat; ++k) f[k] = F[i * kNFeat + k];
    mlp_row_forward<H, B>(sp, f, h1, z, nullptr);
#pragma unroll
    for (int j = 0; j < B; ++j) Z[i * B + j] = z[j];
  }
}

// ---------------------------------------------------------------- loss statistics
// TT = 0 (column form): partial[cta] = [s_j = sum_i z_ij u_ij (B), q_j = sum_i z_ij^2 (B)].
// TT > 0 (subspace form, U is n x TT): partial[cta] = [S_tj = sum_i u_it z_ij (TT x B), q_j (B)].
// SPAN: the second block holds the full Gram M = Z^T Z (B x B) instead of its diagonal q.
template <int TT, int B, bool SPAN = false> struct StatsShape {
  static constexpr int NS = TT == 0 ? B : TT * B;
  static constexpr int NQ = SPAN ? B * B : B;
  static constexpr int NP = NS + NQ;
};

template <int H, int B, int TT, bool SPAN = false>
__global__ void __launch_bounds__(256) mlp_stats_kernel(const float* __restrict__ F, int64_t n,
                                                        const float* __restrict__ params,
                                                        const float* __restrict__ U,
                                                        double* __restrict__ partial) {
  using P = MlpParams<H, B>;
  using SS = StatsShape<TT, B, SPAN>;
  __shared__ float sp[P::COUNT];
  __shared__ double red[SS::NP][8];
  for (int e = threadIdx.x; e < P::COUNT; e += blockDim.x) sp[e] = params[e];
  __syncthreads();
  double s[SS::NS], q[SS::NQ];
#pragma unroll
  for (int j = 0; j < SS::NS; ++j) s[j] = 0.0;
#pragma unroll
  for (int j = 0; j < SS::NQ; ++j) q[j] = 0.0;
#pragma unroll 1
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // keep the weight loads inside the loop (hoisting 64 x 64 shared loads spills registers)
    asm volatile("" ::: "memory");
    float f[kNFeat], h1[H], z[B];
#pragma unroll
    for (int k = 0; k < kNFeat; ++k) f[k] = F[i * kNFeat + k];
    mlp_row_forward<H, B>(sp, f, h1, z, nullptr);
    if (TT == 0) {
#pragma unroll
      for (int j = 0; j < B; ++j) s[j] += (double)z[j] * (double)U[i * B + j];
    } else {
#pragma unroll
      for (int t = 0; t < (TT == 0 ? 1 : TT); ++t) {
        const double u = (double)U[i * (TT == 0 ? 1 : TT) + t];
#pragma unroll
        for (int j = 0; j < B; ++j) s[t * B + j] += u * (double)z[j];
      }
    }
    if (SPAN) {
#pragma unroll
      for (int k = 0; k < B; ++k)
#pragma unroll
        for (int j = 0; j < B; ++j) q[(k * B + j) % SS::NQ] += (double)z[k] * (double)z[j];
    } else {
#pragma unroll
      for (int j = 0; j < B; ++j) q[j] += (double)z[j] * (double)z[j];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < SS::NP; ++j) {
    double v = j < SS::NS ? s[j] : q[j - SS::NS];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[j][warp] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < SS::NP; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[e][w];
    partial[(int64_t)blockIdx.x * SS::NP + e] = t;
  }
}

// ---------------------------------------------------------------- backward
// Tiles of TR rows: each thread runs one row forward and backward and leaves its activations
// and gradients in shared memory; then each thread adds the tile's contribution to the
// gradient entries it owns (entry e = tid + k * TR), so the per-CTA sums are deterministic.
constexpr int kTR = 128;

// Row strides are padded by one float so a warp writing 32 consecutive rows hits 32 banks.
template <int H, int B, int TT, bool SPAN = false>
struct GradSmem {
  static constexpr int LDF = kNFeat + 1, LD = H + 1, LDZ = B + 1;
  static constexpr int F = 0, H1 = F + kTR * LDF, H2 = H1 + kTR * LD, DH1 = H2 + kTR * LD,
                       DH2 = DH1 + kTR * LD, DZ = DH2 + kTR * LD, PAR = DZ + kTR * LDZ,
                       COEF = PAR + MlpParams<H, B>::COUNT,
                       TOTAL = COEF + StatsShape<TT, B, SPAN>::NP;
};

// dz_ij: column form ca_j u_ij + cb_j z_ij; subspace form sum_t u_it A_tj + c_j z_ij, with the
// coefficients (per column, from mlp_loss_coef_kernel) in shared memory.
template <int H, int B, int TT, bool SPAN = false>
__global__ void __launch_bounds__(kTR) mlp_grad_kernel(const float* __restrict__ F, int64_t n,
                                                       const float* __restrict__ params,
                                                       const float* __restrict__ U,
                                                       const double* __restrict__ coef,
                                                       double* __restrict__ partial) {
  using P = MlpParams<H, B>;
  using S = GradSmem<H, B, TT, SPAN>;
  using SS = StatsShape<TT, B, SPAN>;
  constexpr int KPER = (P::COUNT + kTR - 1) / kTR;
  extern __shared__ __align__(16) float sm[];
  float* sp = sm + S::PAR;
  float* sc = sm + S::COEF;
  for (int e = threadIdx.x; e < P::COUNT; e += kTR) sp[e] = params[e];
  for (int e = threadIdx.x; e < SS::NP; e += kTR) sc[e] = (float)coef[e];
  float acc[KPER];
#pragma unroll
  for (int k = 0; k < KPER; ++k) acc[k] = 0.0f;
  const int t = threadIdx.x;
  for (int64_t r0 = (int64_t)blockIdx.x * kTR; r0 < n; r0 += (int64_t)gridDim.x * kTR) {
    const int rows = (int)min((int64_t)kTR, n - r0);
    __syncthreads();  // params loaded / previous tile consumed
    if (t < rows) {
      const int64_t i = r0 + t;
      float f[kNFeat], h1[H], z[B];
#pragma unroll
      for (int k = 0; k < kNFeat; ++k) f[k] = F[i * kNFeat + k];
      mlp_row_forward<H, B>(sp, f, h1, z, sm + S::H2 + t * S::LD);
#pragma unroll
      for (int p = 0; p < H; ++p) sm[S::H1 + t * S::LD + p] = h1[p];
#pragma unroll
      for (int k = 0; k < kNFeat; ++k) sm[S::F + t * S::LDF + k] = f[k];
      float dz[B];
      if (SPAN) {                            // z-term: z C with C (B x B)
#pragma unroll
        for (int j = 0; j < B; ++j) {
          float a = 0.0f;
#pragma unroll
          for (int k = 0; k < B; ++k) a = fmaf(z[k], sc[SS::NS + (k * B + j) % SS::NQ], a);
          dz[j] = a;
        }
      } else {
#pragma unroll
        for (int j = 0; j < B; ++j) dz[j] = sc[SS::NS + j] * z[j];
      }
      if (TT == 0) {
#pragma unroll
        for (int j = 0; j < B; ++j) dz[j] = fmaf(sc[j], U[i * B + j], dz[j]);
      } else {
#pragma unroll
        for (int tt = 0; tt < (TT == 0 ? 1 : TT); ++tt) {
          const float u = U[i * (TT == 0 ? 1 : TT) + tt];
#pragma unroll
          for (int j = 0; j < B; ++j) dz[j] = fmaf(u, sc[tt * B + j], dz[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < B; ++j) sm[S::DZ + t * S::LDZ + j] = dz[j];
      // dh2 = (dz W3^T) * [h2 > 0]
#pragma unroll 1
      for (int q = 0; q < H; ++q) {
        float a = 0.0f;
#pragma unroll
        for (int j = 0; j < B; ++j) a = fmaf(dz[j], sp[P::W3 + q * B + j], a);
        sm[S::DH2 + t * S::LD + q] = sm[S::H2 + t * S::LD + q] > 0.0f ? a : 0.0f;
      }
      // dh1 = (dh2 W2^T) * [h1 > 0]
#pragma unroll 1
      for (int p = 0; p < H; ++p) {
        float a = 0.0f;
#pragma unroll 8
        for (int q = 0; q < H; ++q) a = fmaf(sm[S::DH2 + t * S::LD + q], sp[P::W2 + p * H + q], a);
        sm[S::DH1 + t * S::LD + p] = sm[S::H1 + t * S::LD + p] > 0.0f ? a : 0.0f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPER; ++k) {
      const int e = t + k * kTR;
      if (e >= P::COUNT) continue;
      float a = 0.0f;
      if (e < P::B1) {                       // W1[i][h] += F[r][i] dh1[r][h]
        const int i = e / H, hh = e % H;
        for (int r = 0; r < rows; ++r) a = fmaf(sm[S::F + r * S::LDF + i], sm[S::DH1 + r * S::LD + hh], a);
      } else if (e < P::W2) {                // b1[h] += dh1[r][h]
        const int hh = e - P::B1;
        for (int r = 0; r < rows; ++r) a += sm[S::DH1 + r * S::LD + hh];
      } else if (e < P::B2) {                // W2[p][q] += h1[r][p] dh2[r][q]
        const int p = (e - P::W2) / H, q = (e - P::W2) % H;
        for (int r = 0; r < rows; ++r) a = fmaf(sm[S::H1 + r * S::LD + p], sm[S::DH2 + r * S::LD + q], a);
      } else if (e < P::W3) {                // b2[q] += dh2[r][q]
        const int q = e - P::B2;
        for (int r = 0; r < rows; ++r) a += sm[S::DH2 + r * S::LD + q];
      } else if (e < P::B3) {                // W3[q][j] += h2[r][q] dz[r][j]
        const int q = (e - P::W3) / B, j = (e - P::W3) % B;
        for (int r = 0; r < rows; ++r) a = fmaf(sm[S::H2 + r * S::LD + q], sm[S::DZ + r * S::LDZ + j], a);
      } else {                               // b3[j] += dz[r][j]
        const int j = e - P::B3;
        for (int r = 0; r < rows; ++r) a += sm[S::DZ + r * S::LDZ + j];
      }
      acc[k] += a;
    }
  }
#pragma unroll
  for (int k = 0; k < KPER; ++k) {
    const int e = t + k * kTR;
    if (e < P::COUNT) partial[(int64_t)blockIdx.x * P::COUNT + e] = (double)acc[k];
  }
}

__global__ void grad_reduce_kernel(const double* __restrict__ partial, int nctas, int count,
                                   float* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double s = 0.0;
  for (int c = 0; c < nctas; ++c) s += partial[(int64_t)c * count + e];
  grad[e] = (float)s;
}

// From the per-CTA partials (added in CTA order): T = 0 (column form) coef = [-2 s_j/q_j (B),
// 2 s_j^2/q_j^2 (B)], L = sum_j (1 - s_j^2/q_j); T > 0 (subspace form) coef = [-2 S_tj/q_j
// (T x B), 2 P_j/q_j^2 (B)] with P_j = sum_t S_tj^2, L = sum_j (1 - P_j/q_j).
__global__ void loss_coef_kernel(const double* __restrict__ partial, int nctas, int B, int T,
                                 double* __restrict__ coef, double* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  const int ns = T == 0 ? B : T * B, np = ns + B;
  double L = 0.0;
  for (int j = 0; j < B; ++j) {
    double q = 0.0;
    for (int c = 0; c < nctas; ++c) q += partial[(int64_t)c * np + ns + j];
    const int rows = T == 0 ? 1 : T;
    double P = 0.0;
    for (int t = 0; t < rows; ++t) {
      double st = 0.0;
      const int idx = T == 0 ? j : t * B + j;
      for (int c = 0; c < nctas; ++c) st += partial[(int64_t)c * np + idx];
      P += st * st;
      coef[idx] = q > 0.0 ? -2.0 * st / q : 0.0;
    }
    coef[ns + j] = q > 0.0 ? 2.0 * P / (q * q) : 0.0;
    L += q > 0.0 ? 1.0 - P / q : 1.0;
  }
  *loss = L;
}

// Span form: from partials [S (T x B), M (B x B)]: N = S^T S, Mi = M^{-1} (Gauss-Jordan with
// partial pivoting, B <= 8), coef = [A = -2 S Mi (T x B), C = 2 Mi N Mi (B x B)],
// loss = B - tr(Mi N).
__global__ void span_coef_kernel(const double* __restrict__ partial, int nctas, int B, int T,
                                 double* __restrict__ coef, double* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  const int ns = T * B, np = ns + B * B;
  double S[16 * 8], M[8 * 8], Mi[8 * 8], N[8 * 8], X[8 * 8];
  for (int e = 0; e < np; ++e) {
    double v = 0.0;
    for (int c = 0; c < nctas; ++c) v += partial[(int64_t)c * np + e];
    if (e < ns) S[e] = v;
    else M[e - ns] = v;
  }
  for (int e = 0; e < B * B; ++e) Mi[e] = (e / B == e % B) ? 1.0 : 0.0;
  bool ok = true;
  for (int c = 0; c < B && ok; ++c) {
    int piv = c;
    for (int r = c + 1; r < B; ++r)
      if (fabs(M[r * B + c]) > fabs(M[piv * B + c])) piv = r;
    if (!(fabs(M[piv * B + c]) > 0.0)) { ok = false; break; }
    for (int k = 0; k < B; ++k) {
      double t = M[c * B + k]; M[c * B + k] = M[piv * B + k]; M[piv * B + k] = t;
      t = Mi[c * B + k]; Mi[c * B + k] = Mi[piv * B + k]; Mi[piv * B + k] = t;
    }
    const double d = M[c * B + c];
    for (int k = 0; k < B; ++k) { M[c * B + k] /= d; Mi[c * B + k] /= d; }
    for (int r = 0; r < B; ++r) {
      if (r == c) continue;
      const double f = M[r * B + c];
      for (int k = 0; k < B; ++k) { M[r * B + k] -= f * M[c * B + k]; Mi[r * B + k] -= f * Mi[c * B + k]; }
    }
  }
  if (!ok) {
    for (int e = 0; e < np; ++e) coef[e] = 0.0;
    *loss = (double)B;
    return;
  }
  for (int i = 0; i < B; ++i)                       // N = S^T S
    for (int j = 0; j < B; ++j) {
      double v = 0.0;
      for (int t = 0; t < T; ++t) v += S[t * B + i] * S[t * B + j];
      N[i * B + j] = v;
    }
  double tr = 0.0;
  for (int i = 0; i < B; ++i)                       // X = Mi N, tr(Mi N)
    for (int j = 0; j < B; ++j) {
      double v = 0.0;
      for (int k = 0; k < B; ++k) v += Mi[i * B + k] * N[k * B + j];
      X[i * B + j] = v;
      if (i == j) tr += v;
    }
  for (int t = 0; t < T; ++t)                       // A = -2 S Mi
    for (int j = 0; j < B; ++j) {
      double v = 0.0;
      for (int k = 0; k < B; ++k) v += S[t * B + k] * Mi[k * B + j];
      coef[t * B + j] = -2.0 * v;
    }
  for (int i = 0; i < B; ++i)                       // C = 2 (Mi N) Mi
    for (int j = 0; j < B; ++j) {
      double v = 0.0;
      for (int k = 0; k < B; ++k) v += X[i * B + k] * Mi[k * B + j];
      coef[ns + i * B + j] = 2.0 * v;
    }
  *loss = (double)B - tr;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// ---------------------------------------------------------------- dispatch
template <int H, int B>
static int forward_hb(const float* F, int64_t n, const float* params, float* Z, cudaStream_t s) {
  const int ctas = (int)std::min<int64_t>(ceil_div(n, 256), 4 * num_sms());
  mlp_forward_kernel<H, B><<<std::max(ctas, 1), 256, 0, s>>>(F, n, params, Z);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

template <int H, int B, int TT = 0, bool SPAN = false>
static int loss_grad_hb(const float* F, int64_t n, const float* params, const float* U,
                        float* grad, double* loss_host, cudaStream_t s) {
  using P = MlpParams<H, B>;
  using S = GradSmem<H, B, TT, SPAN>;
  using SS = StatsShape<TT, B, SPAN>;
  const int sctas = std::max(1, (int)std::min<int64_t>(ceil_div(n, 256), 2 * num_sms()));
  const int gctas = std::max(1, (int)std::min<int64_t>(ceil_div(n, kTR), num_sms()));
  double* part = small_scratch(15, (size_t)sctas * SS::NP + SS::NP + 1);
  double* gpart = small_scratch(16, (size_t)gctas * P::COUNT);
  if (!part || !gpart) return FE_ERR_OOM;
  double* coef = part + (size_t)sctas * SS::NP;
  double* dloss = coef + SS::NP;
  mlp_stats_kernel<H, B, TT, SPAN><<<sctas, 256, 0, s>>>(F, n, params, U, part);
  count_launch();
  if (SPAN) span_coef_kernel<<<1, 32, 0, s>>>(part, sctas, B, TT, coef, dloss);
  else loss_coef_kernel<<<1, 32, 0, s>>>(part, sctas, B, TT, coef, dloss);
  count_launch();
  const size_t smem = sizeof(float) * S::TOTAL;
  FE_ARG(smem <= 220 * 1024, "mlp: hidden/b too large for the gradient kernel");
  static KernelSetup ks;
  FE_TRY(kernel_configure(ks, reinterpret_cast<const void*>(mlp_grad_kernel<H, B, TT, SPAN>), (int)smem));
  mlp_grad_kernel<H, B, TT, SPAN><<<gctas, kTR, smem, s>>>(F, n, params, U, coef, gpart);
  count_launch();
  grad_reduce_kernel<<<(unsigned)ceil_div(P::COUNT, 256), 256, 0, s>>>(gpart, gctas, P::COUNT, grad);
  count_launch();
  FE_CUDA(cudaGetLastError());
  if (loss_host) {
    FE_CUDA(cudaMemcpyAsync(loss_host, dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
  }
  return FE_OK;
}

#define FE_MLP_DISPATCH(H, EXPR_B)                                   \
  switch (b) {                                                       \
    case 1: return EXPR_B(H, 1);                                     \
    case 2: return EXPR_B(H, 2);                                     \
    case 4: return EXPR_B(H, 4);                                     \
    case 8: return EXPR_B(H, 8);                                     \
    case 16: return EXPR_B(H, 16);                                   \
  }

int mlp_forward(const float* F, int64_t n, const float* params, int hidden, int b, float* Z,
                cudaStream_t s) {
#define FWD(H, B) forward_hb<H, B>(F, n, params, Z, s)
  if (hidden == 64) { FE_MLP_DISPATCH(64, FWD) }
  if (hidden == 32) { FE_MLP_DISPATCH(32, FWD) }
#undef FWD
  return set_error(FE_ERR_INVALID, "mlp: hidden must be 32 or 64 and b in {1,2,4,8,16} (got %d, %d)", hidden, b);
}

int mlp_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                  const float* U, float* grad, double* loss, cudaStream_t s) {
#define LG(H, B) loss_grad_hb<H, B>(F, n, params, U, grad, loss, s)
  if (hidden == 64) { FE_MLP_DISPATCH(64, LG) }
  if (hidden == 32) { FE_MLP_DISPATCH(32, LG) }
#undef LG
  return set_error(FE_ERR_INVALID, "mlp: hidden must be 32 or 64 and b in {1,2,4,8,16} (got %d, %d)", hidden, b);
}

int mlp_subspace_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                           const float* U, int t, float* grad, double* loss, cudaStream_t s) {
#define SLG(TT, B) loss_grad_hb<64, B, TT>(F, n, params, U, grad, loss, s)
  if (hidden == 64 && (b == 4 || b == 8) && (t == 4 || t == 8 || t == 16)) {
    if (b == 4) {
      if (t == 4) return SLG(4, 4);
      if (t == 8) return SLG(8, 4);
      return SLG(16, 4);
    }
    if (t == 4) return SLG(4, 8);
    if (t == 8) return SLG(8, 8);
    return SLG(16, 8);
  }
#undef SLG
  return set_error(FE_ERR_INVALID, "mlp subspace loss: needs hidden 64, b in {4, 8}, t in {4, 8, 16} (got %d, %d, %d)", hidden, b, t);
}

int mlp_span_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                       const float* U, int t, float* grad, double* loss, cudaStream_t s) {
#define PLG(TT, B) loss_grad_hb<64, B, TT, true>(F, n, params, U, grad, loss, s)
  if (hidden == 64 && b == 4 && t == 4) return PLG(4, 4);
  if (hidden == 64 && b == 4 && t == 8) return PLG(8, 4);
  if (hidden == 64 && b == 8 && t == 8) return PLG(8, 8);
#undef PLG
  return set_error(FE_ERR_INVALID, "mlp span loss: needs hidden 64 and (b, t) in {(4,4), (4,8), (8,8)} (got %d, %d, %d)", hidden, b, t);
}

// Start block for fe_eigs: features -> MLP -> FP64 row-major n x b (the solver orthonormalises).
int mlp_start_block(fe_csr h, const float* weights, int hidden, int b, uint64_t seed,
                    double* out, cudaStream_t s) {
  const int64_t n = h->n;
  DevBuf fbuf, zbuf;
  FE_TRY(fbuf.alloc(sizeof(float) * (size_t)n * kNFeat));
  FE_TRY(zbuf.alloc(sizeof(float) * (size_t)n * b));
  FE_TRY(vertex_features(h, seed, fbuf.as<float>(), s));
  FE_TRY(mlp_forward(fbuf.as<float>(), n, weights, hidden, b, zbuf.as<float>(), s));
  FE_TRY(convert_block(zbuf.p, FE_F32, b, out, FE_F64, b, n, b, s));
  FE_CUDA(cudaStreamSynchronize(s));
  return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

int64_t fe_mlp_param_count(int hidden, int b) {
  if ((hidden != 32 && hidden != 64) || !is_pow2_le16(b)) return -1;
  return mlp_param_count(hidden, b);
}

int fe_vertex_features(fe_csr h, uint64_t seed, float* F) {
  FE_ARG(h && F, "fe_vertex_features: NULL argument");
  return vertex_features(h, seed, F, cur_stream());
}

int fe_mlp_forward(const float* F, int64_t n, const float* params, int hidden, int b, float* Z) {
  FE_ARG(F && params && Z && n >= 1, "fe_mlp_forward: bad argument");
  return mlp_forward(F, n, params, hidden, b, Z, cur_stream());
}

int fe_mlp_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                     const float* U, float* grad, double* loss) {
  FE_ARG(F && params && U && grad && n >= 1, "fe_mlp_loss_grad: bad argument");
  return mlp_loss_grad(F, n, params, hidden, b, U, grad, loss, cur_stream());
}

int fe_mlp_subspace_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                              const float* U, int t, float* grad, double* loss) {
  FE_ARG(F && params && U && grad && n >= 1, "fe_mlp_subspace_loss_grad: bad argument");
  return mlp_subspace_loss_grad(F, n, params, hidden, b, U, t, grad, loss, cur_stream());
}

int fe_mlp_span_loss_grad(const float* F, int64_t n, const float* params, int hidden, int b,
                          const float* U, int t, float* grad, double* loss) {
  FE_ARG(F && params && U && grad && n >= 1, "fe_mlp_span_loss_grad: bad argument");
  return mlp_span_loss_grad(F, n, params, hidden, b, U, t, grad, loss, cur_stream());
}

int fe_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count, double lr,
                double beta1, double beta2, double eps, int step) {
  FE_ARG(params && grad && m && v && count >= 1 && step >= 1, "fe_mlp_adam: bad argument");
  const float c1 = 1.0f - (float)pow(beta1, step), c2 = 1.0f - (float)pow(beta2, step);
  const int ctas = (int)std::min<int64_t>(ceil_div(count, 256), 4 * num_sms());
  adam_kernel<<<std::max(ctas, 1), 256, 0, cur_stream()>>>(params, grad, m, v, count, (float)lr,
                                                          (float)beta1, (float)beta2, (float)eps, c1, c2);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

}  // extern "C"
