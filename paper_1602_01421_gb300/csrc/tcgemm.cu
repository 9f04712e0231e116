// FP64 tall-skinny products on the FP16 tensor cores by exact digit splitting ("split
// products"; the Ozaki scheme, Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012), for
// the restart / Ritz-vector product of the Block Krylov-Schur solver (Table 1 "op1" shape,
// V_out = V Y with V n x K, Y K x N, K <= 64 and N <= 32):
//
//   * every V row is scaled by its largest binary exponent and its 53-bit aligned significands
//     are cut into seven 8-bit digits (sign-magnitude, so every digit is an integer in
//     [-255, 255] and exact in FP16): V[r][c] = 2^(Er - 1075) sum_i d_i[r][c] 2^(45 - 8 i);
//   * every Y column likewise by its largest exponent: Y[c][q] = 2^(Fq - 1075) sum_j e_j 2^(45-8j);
//   * the digit products are exact in the tensor core's FP32 accumulator as long as each
//     accumulator sums at most 2^24 / 255^2 = 258 of them: one accumulator per digit-weight
//     class g = i + j (g <= 6) and per 32-wide slice of K holds at most 7 * 32 products;
//   * V Y = 2^(Er + Fq - 2108) * T with T = sum_g D_g 2^(8 (6 - g)), assembled in 64-bit
//     integer arithmetic from the accumulators (T / 2^12, exact up to the dropped bits) and
//     rounded once (truncation) to FP64.
//
// Error: the digit products dropped (i + j >= 7), the truncation of each entry below its
// row's (column's) leading bit and the 12 dropped bits of T bound |error| <=
// 2^-49 (K + 1) max_c |V[r][c]| max_c |Y[c][q]| + 2^-52 |result|; the FP64 pipe is not used at
// all (FP64 on this part runs at 1/64 of FP32).
//
// Kernels: for K <= 32 a warp-specialised pipeline (tc_combine_pipe_kernel: TMA producer,
// digit splitters, one MMA-issuing thread, result assemblers over double-buffered tiles; see its
// comment); for 32 < K <= 64 tc_combine_kernel, one 128-row tile per loop trip and two
// persistent CTAs of 256 threads per SM: two threads share a row of the V tile, each splits half
// of its K values into the digit tiles, thread 0 issues one MMA per digit and K-step and commits
// to an mbarrier, then the two threads assemble half of the row's N results each.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "fe_internal.cuh"
#include "tc.cuh"
#include "vec.cuh"

namespace fe {

namespace {

constexpr int kDigits = 7;           // 8-bit digits per 53-bit significand (7 * 8 >= 53)
constexpr int kClasses = 7;          // digit-weight classes g = i + j kept (g <= 6)
constexpr int kTileRows = 128;       // MMA M
constexpr int kKChunk = 32;          // K columns per accumulator set (exactness bound)
constexpr int kMaxK = 64;
constexpr int kMaxN = 32;
constexpr int kThreads = 256;
// Sleeping waits: at most 2^16 polls of up to 32 us each (about 2 s in all).
constexpr uint32_t kPipePolls = 1u << 16;
constexpr uint32_t kPipeSleepNs = 32768;
constexpr int kCoreBytes = 128;      // 8 rows x 16 bytes
// A (V digits): per (K chunk, digit) a 128 x 32 FP16 tile = 8 KB; SBO = 4 core matrices
constexpr int kATileBytes = kTileRows * kKChunk * 2;
constexpr uint32_t kLBO = kCoreBytes;               // next core matrix along K
constexpr uint32_t kSBO = (kKChunk / 8) * kCoreBytes;  // next 8-row group

// Byte offset of element (row, k) of a [rows x 32] 16-bit K-major tile (k < 32).
__host__ __device__ inline uint32_t tile_off(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// Biased exponent field of a double (0 for zero and subnormals, which are read as zero).
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// Significand of x aligned to the binary exponent field emax (>= x's): a non-negative integer
// below 2^53 with x = +-M * 2^(emax - 1075) up to the bits shifted out.
__device__ __forceinline__ uint64_t aligned_sig(double x, int emax) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const int sh = emax - e;
  if (e == 0 || sh > 52) return 0;
  return ((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> sh;
}

// Digit i of an aligned significand: bits [45 - 8 i, 52 - 8 i] for i < 6, the low 5 bits
// shifted up by 3 for i = 6 (weight 2^(45 - 8 i) in both cases).
__device__ __forceinline__ uint32_t digit(uint64_t m, int i) {
  return i < 6 ? (uint32_t)(m >> (45 - 8 * i)) & 0xFFu : ((uint32_t)m & 0x1Fu) << 3;
}

// The aligned significand shifted up by 3 bits (56 bits): digit i is then byte 6 - i.
__device__ __forceinline__ uint64_t aligned_sig56(double x, int emax) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const int sh = emax - e;
  if (e == 0 || sh > 52) return 0;
  return (((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 3) >> sh;
}

// FP16 x2 fused multiply-add on packed halves (round to nearest).
__device__ __forceinline__ uint32_t hfma2_u32(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(y), "r"(z));
  return d;
}

// The seven digits of two FP64 values x0, x1 relative to the exponent field emax (>= theirs),
// as packed FP16 pairs: w[i][e] holds digit i of x0 (low half) and of x1 (high half), each with
// its value's sign.  Per digit pair: a byte permute takes the two digit bytes of the 56-bit
// significands, a LOP3 puts each under the FP16 exponent of 1024 (1024 + d is exact for
// d < 1024), and one FP16 FMA forms (1024 + d) s - 1024 s = s d exactly (s = +-1).
__device__ __forceinline__ void split_pair_f16(double x0, double x1, int emax, uint32_t (&w)[kDigits][4],
                                               int e) {
  const uint64_t m0 = aligned_sig56(x0, emax), m1 = aligned_sig56(x1, emax);
  const uint32_t h0 = (uint32_t)((uint64_t)__double_as_longlong(x0) >> 32);
  const uint32_t h1 = (uint32_t)((uint64_t)__double_as_longlong(x1) >> 32);
  const uint32_t s2 = 0x3C003C00u | ((h0 >> 16) & 0x8000u) | (h1 & 0x80000000u);  // (+-1, +-1)
  const uint32_t c2 = s2 ^ 0xD800D800u;                                          // -1024 (+-1)
#pragma unroll
  for (int i = 0; i < kDigits; ++i) {
    const int k = 6 - i;   // byte of the 56-bit significand holding digit i
    const uint32_t lo0 = (uint32_t)m0, hi0 = (uint32_t)(m0 >> 32);
    const uint32_t lo1 = (uint32_t)m1, hi1 = (uint32_t)(m1 >> 32);
    const uint32_t pa = k < 4 ? lo0 : hi0, pb = k < 4 ? lo1 : hi1;
    const uint32_t sel = (uint32_t)((k & 3) | ((4 + (k & 3)) << 8));
    const uint32_t r = (__byte_perm(pa, pb, sel) & 0x00FF00FFu) | 0x64006400u;
    w[i][e] = hfma2_u32(r, s2, c2);
  }
}

// The FP16 bits of s d for a digit d in [0, 255] and a sign bit (the same exact FMA).
__device__ __forceinline__ uint16_t digit_f16(uint32_t d, uint32_t sign) {
  const uint32_t s2 = 0x3C00u | (sign << 15);
  return (uint16_t)(hfma2_u32(0x6400u | d, s2, s2 ^ 0xD800u) & 0xFFFFu);
}

// Exact integer value of an FP32 accumulator holding an integer of magnitude below 2^24.
__device__ __forceinline__ int32_t acc_int(uint32_t bits) {
  return __float2int_rn(__uint_as_float(bits));
}

// The accumulated T = hi 2^32 + lo (|hi| < 2^40, |lo| < 2^50) is taken as floor(T / 2^12), an
// int64 of at most 60 bits, before it is rounded to FP64: the 12 dropped bits are below the
// digit truncation already made (2^-50 of max|V_r| max|Y_q|).
constexpr int kAsmShift = 12;

// 2^s * (hi 2^20 + floor(lo / 2^12)) truncated to FP64; zero below the normal range, infinity
// above it.  Integer operations only, without branches.
__device__ __forceinline__ double assemble(int64_t hi, int64_t lo, int s) {
  const int64_t t = (hi << (32 - kAsmShift)) + (lo >> kAsmShift);
  const uint64_t sign = (uint64_t)t & 0x8000000000000000ull;
  const uint64_t a = t < 0 ? (uint64_t)(-t) : (uint64_t)t;
  const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
  const int lz = ah != 0 ? __clz(ah) : 32 + __clz(al);  // 64 when a == 0 (32-bit counts)
  const uint64_t m = a << (lz & 63);                    // leading one at bit 63
  const int ef = 63 - lz + s + 1023;
  uint64_t bits = sign | ((uint64_t)(uint32_t)ef << 52) | ((m >> 11) & 0xFFFFFFFFFFFFFull);
  bits = (a == 0 || ef <= 0) ? sign : bits;
  bits = ef >= 2047 ? (sign | 0x7FF0000000000000ull) : bits;
  return __longlong_as_double((long long)bits);
}

// Bounded wait that sleeps until the phase completes: waiting threads take no issue slots from
// the other CTA on the SM.  True when the phase completed.
__device__ __forceinline__ bool wait_sleep(uint64_t* bar, uint32_t parity) {
  return tc::mbar_wait(bar, parity, 1) || tc::mbar_wait_sleep(bar, parity, kPipePolls, kPipeSleepNs);
}

struct TcArgs {
  const double* vblk[kMaxK];   // K / BV blocks of n x BV (ld BV)
  double* oblk[kMaxN];         // N / BV output blocks of n x BV (ld BV); fewer when BV < 4
  int64_t n;
  int K, N, NP;                // NP: N padded to the MMA's N (16 or 32)
  int nkc;                     // K chunks of 32
  const uint16_t* bdig;        // global: [nkc][7][NP x 32] canonical tiles
  const int* fexp;             // global: N column exponent fields of Y
  int* status;                 // device word: 1 = an MMA wait ran out
  double beta;                 // Out = beta Out + (alpha V Y); beta = 0: Out is not read
  int bulk;                    // 1: every V block is 16-byte aligned (TMA bulk copies allowed)
  int ovec;                    // 1: every output block is 16-byte aligned (vector stores allowed)
};

}  // namespace

// Y (K x N FP64, row-major, ld ldy) -> per-column exponent fields and the seven digit tiles of
// every 32-row K chunk in the MMA's B layout (row q of B = column q of Y; rows N..NP-1 and
// K beyond K zero).  One CTA.
__global__ void tc_prep_y_kernel(const double* __restrict__ Y, int ldy, double alpha, int K, int N, int NP,
                                 int nkc, uint16_t* __restrict__ bdig, int* __restrict__ fexp) {
  __shared__ int sf[kMaxN];
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    int f = 0;
    for (int c = 0; c < K; ++c) f = max(f, exp_field(alpha * Y[c * ldy + q]));
    sf[q] = f;
    fexp[q] = f;
  }
  __syncthreads();
  const int per_tile = NP * kKChunk;  // elements of one [NP x 32] tile
  const int total = nkc * per_tile;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int kc = e / per_tile, r = e % per_tile;
    const int q = r / kKChunk, k = r % kKChunk;
    const int c = kc * kKChunk + k;
    uint64_t m = 0;
    uint32_t sgn = 0;
    if (q < N && c < K) {
      const double y = alpha * Y[c * ldy + q];
      m = aligned_sig(y, sf[q]);
      sgn = (uint32_t)((uint64_t)__double_as_longlong(y) >> 63);
    }
    for (int j = 0; j < kDigits; ++j) {
      const uint16_t bits = digit_f16(digit(m, j), sgn);
      char* tile = reinterpret_cast<char*>(bdig) + (size_t)(kc * kDigits + j) * per_tile * 2;
      *reinterpret_cast<uint16_t*>(tile + tile_off(q, k)) = bits;
    }
  }
}

// Row r of a 128-row tile is handled by two threads (warps w and w + 4 address the same TMEM
// lane quarter): each loads and splits half of the row's K values, and each assembles half of
// the row's N results.
// K <= 32: two CTAs per SM (256 TMEM columns each); K <= 64: one (512 columns).
template <int BV, int KMAX>
__global__ void __launch_bounds__(kThreads, KMAX <= 32 ? 2 : 1) tc_combine_kernel(const TcArgs a) {
  constexpr int KH = KMAX / 2;  // V values per thread
  extern __shared__ __align__(1024) unsigned char smem[];
  const int nkc = a.nkc, NP = a.NP;
  unsigned char* sA = smem;                                        // [nkc][7] x 8 KB
  unsigned char* sB = sA + (size_t)nkc * kDigits * kATileBytes;    // [nkc][7] x NP*64
  const size_t btile = (size_t)NP * kKChunk * 2;
  double* sV = reinterpret_cast<double*>(sB + (size_t)nkc * kDigits * btile);  // [K/BV][128][BV]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sV + (size_t)kTileRows * KMAX);
  uint64_t* lbar = bar + 1;                      // V tile copies
  uint64_t* sDesc = bar + 2;                     // [nkc][7][2] A and B descriptors (K-step 0)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sDesc + 2 * kDigits * (KMAX / kKChunk) * 2);
  int* sF = reinterpret_cast<int*>(tslot + 1);   // N column exponents of Y
  int* sE = sF + kMaxN;                          // [2][128] partial row exponents
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = warp >> 2;
  const int row = (warp & 3) * 32 + lane;        // row of the tile = TMEM lane
  const uint32_t ncols = (uint32_t)nkc * kClasses * NP <= 256 ? 256u : 512u;

  // B digits and column exponents (once per CTA)
  {
    const int4* src = reinterpret_cast<const int4*>(a.bdig);
    int4* dst = reinterpret_cast<int4*>(sB);
    const int n16 = (int)((size_t)nkc * kDigits * btile / 16);
    for (int e = tid; e < n16; e += kThreads) dst[e] = src[e];
    for (int q = tid; q < a.N; q += kThreads) sF[q] = a.fexp[q];
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, ncols);
    tc::tmem_relinquish();
  }
  const int nblk = a.K / BV;
  const bool add_out = a.beta != 0.0;   // decided once: an FP64 compare per result would
                                        // occupy the FP64 pipe
  const int64_t ntiles = (a.n + kTileRows - 1) / kTileRows;
  // a tile's V rows come in by TMA bulk copies (one per block) when their byte count is a
  // multiple of 16 (every full tile); otherwise (a ragged last tile) by plain loads
  auto bulk_ok = [&](int64_t t) {
    return a.bulk && ((uint64_t)min((int64_t)kTileRows, a.n - t * kTileRows) * BV * 8) % 16 == 0;
  };
  auto issue = [&](int64_t t) {
    const int64_t r0 = t * kTileRows;
    const uint32_t bytes = (uint32_t)(min((int64_t)kTileRows, a.n - r0) * BV * 8);
    tc::mbar_arrive_expect_tx(lbar, bytes * (uint32_t)nblk);
    for (int j = 0; j < nblk; ++j) tc::bulk_g2s(sV + (size_t)j * kTileRows * BV, a.vblk[j] + r0 * BV, bytes, lbar);
  };
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_init(lbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0 && (int64_t)blockIdx.x < ntiles && bulk_ok(blockIdx.x)) issue(blockIdx.x);
  const uint32_t tbase = *tslot;
  const uint32_t sa0 = tc::smem_addr(sA), sb0 = tc::smem_addr(sB);
  if (tid == 0)
    for (int kc = 0; kc < nkc; ++kc)
      for (int i = 0; i < kDigits; ++i) {
        sDesc[(kc * kDigits + i) * 2] = tc::smem_desc(sa0 + (uint32_t)((kc * kDigits + i) * kATileBytes), kLBO, kSBO);
        sDesc[(kc * kDigits + i) * 2 + 1] = tc::smem_desc(sb0 + (uint32_t)((kc * kDigits + i) * btile), kLBO, kSBO);
      }
  const int cbeg = half * KH;                    // this thread's first V column
  const int kc_mine = cbeg / kKChunk, k_mine = cbeg % kKChunk;
  uint32_t phase = 0, lphase = 0;
  bool failed = false;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r = tile * kTileRows + row;
    const bool live = r < a.n;
    const bool bulk = bulk_ok(tile);
    bool ok = true;
    if (bulk) {
      ok = wait_sleep(lbar, lphase);
      if (!ok) {
        failed = true;
        wait_sleep(lbar, lphase);  // no copy left in flight
      }
      lphase ^= 1;
    }
    // ---- this thread's half of row r and its largest exponent
    double v[KH];
    int emax = 0;
#pragma unroll
    for (int c0 = 0; c0 < KH; c0 += BV) {
      if (live && cbeg + c0 < a.K) {
        if (bulk) {
          const double* src = sV + ((size_t)((cbeg + c0) / BV) * kTileRows + row) * BV;
#pragma unroll
          for (int p = 0; p < BV; ++p) v[c0 + p] = src[p];
        } else {
          const double* src = a.vblk[(cbeg + c0) / BV] + r * BV;   // scalar loads: any alignment
#pragma unroll
          for (int p = 0; p < BV; ++p) v[c0 + p] = src[p];
        }
      } else {
#pragma unroll
        for (int p = 0; p < BV; ++p) v[c0 + p] = 0.0;
      }
    }
#pragma unroll
    for (int c = 0; c < KH; ++c) emax = max(emax, exp_field(v[c]));
    sE[half * kTileRows + row] = emax;
    __syncthreads();  // every thread has its V values: the staging buffer takes the next tile
    if (tid == 0) {
      const int64_t nt = tile + gridDim.x;
      if (nt < ntiles && bulk_ok(nt)) issue(nt);
    }
    emax = max(sE[row], sE[kTileRows + row]);
    // ---- split into seven digits and write them to the A tiles
#pragma unroll
    for (int k8 = 0; k8 < KH; k8 += 8) {
      uint32_t w[kDigits][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const double x0 = v[k8 + 2 * e], x1 = v[k8 + 2 * e + 1];
        split_pair_f16(x0, x1, emax, w, e);
      }
      const int kk = k_mine + k8;   // column within the chunk
      const int kc = kc_mine + kk / kKChunk;
#pragma unroll
      for (int i = 0; i < kDigits; ++i)
        *reinterpret_cast<uint4*>(sA + (size_t)(kc * kDigits + i) * kATileBytes + tile_off(row, kk % kKChunk)) =
            make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // ---- one thread issues the digit products: class g = i + j accumulates A_i B_j
    if (tid == 0) {
      tc::fence_after_sync();
      // descriptor of K-step ks = that of K-step 0 with the start address advanced by 2 core
      // matrices (256 bytes, 16 in the descriptor's address field)
      // digit i of A against the B digit tiles 0..6-i of the chunk stacked as one operand of
      // (7-i) NP rows: column block j of the product accumulates into class i + j
      for (int kc = 0; kc < nkc; ++kc)
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
          const uint64_t ad = sDesc[(kc * kDigits + i) * 2];
          const uint64_t bd = sDesc[(kc * kDigits) * 2 + 1];
          const uint32_t dt = tbase + (uint32_t)((kc * kClasses + i) * NP);
          const uint32_t id = tc::idesc_f16_f32(kTileRows, (kDigits - i) * NP);
#pragma unroll
          for (int ks = 0; ks < kKChunk / 16; ++ks)
            tc::mma_f16(dt, ad + (uint64_t)(ks * 2 * kLBO >> 4), bd + (uint64_t)(ks * 2 * kLBO >> 4), id,
                         (i > 0 || ks > 0) ? 1u : 0u);
        }
      tc::mma_commit(bar);
    }
    // ---- wait for the products (bounded), then read row `row`'s accumulators
    if (!wait_sleep(bar, phase)) {
      ok = false;
      failed = true;
      wait_sleep(bar, phase);  // let the MMAs in flight finish before TMEM is reused
    }
    phase ^= 1;
    tc::fence_after_sync();
    const uint32_t lane_addr = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    const int ebase = emax - 2108 + kAsmShift;
    for (int q0 = 4 * half; q0 < a.N; q0 += 8) {   // groups of 4 results, alternating halves
      uint32_t acc[KMAX / kKChunk][kClasses][4];
#pragma unroll
      for (int kc = 0; kc < KMAX / kKChunk; ++kc)
        if (kc < nkc)
#pragma unroll
          for (int g = 0; g < kClasses; ++g)
            tc::tmem_ld4(lane_addr + (uint32_t)((kc * kClasses + g) * NP + q0), acc[kc][g]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int kc = 0; kc < KMAX / kKChunk; ++kc)
        if (kc < nkc)
#pragma unroll
          for (int g = 0; g < kClasses; ++g) tc::reg_after_wait(acc[kc][g]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u;
        int64_t hi = 0, lo = 0;
#pragma unroll
        for (int kc = 0; kc < KMAX / kKChunk; ++kc)
          if (kc < nkc) {
            // 32 x 32 -> 64-bit multiply-adds by powers of two
            hi += (int64_t)acc_int(acc[kc][0][u]) * 65536 + (int64_t)acc_int(acc[kc][1][u]) * 256 +
                  (int64_t)acc_int(acc[kc][2][u]);
            lo += (int64_t)acc_int(acc[kc][3][u]) * 16777216 + (int64_t)acc_int(acc[kc][4][u]) * 65536 +
                  (int64_t)acc_int(acc[kc][5][u]) * 256 + (int64_t)acc_int(acc[kc][6][u]);
          }
        if (live && q < a.N) {
          double y = 0.0;
          if (!ok) y = __longlong_as_double(0x7FF8000000000000ll);
          else if (emax > 0) y = assemble(hi, lo, ebase + sF[q]);
          double* dst = a.oblk[q / BV] + r * BV + q % BV;
          if (add_out) y = fma(a.beta, *dst, y);
          *dst = y;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM read, A tiles and row exponents free for the next tile
  }
  if (failed && lane == 0) atomicExch(a.status, 1);
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// Shared-memory bytes of tc_combine_kernel for nkc K chunks and padded N.
static size_t tc_smem_bytes(int nkc, int NP) {
  const int kmax = nkc == 1 ? 32 : 64;
  return (size_t)nkc * kDigits * kATileBytes + (size_t)nkc * kDigits * NP * kKChunk * 2 +
         (size_t)kTileRows * kmax * 8 + 16 + 8 * 2 * kDigits * (kmax / kKChunk) * 2 + 8 + 4 * kMaxN +
         4 * 2 * kTileRows + 64;
}

// ---------------------------------------------------------------- pipelined form (K <= 32)
// The same product with the phases of consecutive tiles overlapped.  One persistent CTA per SM
// with four warp roles:
//   warps 0-7   split V rows into digits: a unit is 8 columns of one row, unit u = row
//               + 128 cb (cb < ceil(K / 8)), thread t takes units t and t + 256, so the work
//               follows K; units write the digit tiles of buffer t % 2;
//   warp 16     (one thread) issues the TMA copies of tile t's V rows into staging buffer t % 2;
//   warp 17     (one thread) issues tile t's MMAs into TMEM buffer t % 2 and owns the TMEM
//               allocation;
//   warps 8-15  read tile t's accumulators (TMEM lane quarter = warp % 4, two threads per row,
//               alternate groups of four results), assemble and store them; with beta != 0 and
//               N <= 16 the rows of Out for tile t + 1 are loaded while tile t is assembled.
// V staging, digit tiles and accumulators are double-buffered, so tile t + 1 is split while tile
// t's products run and its results are assembled.  Five mbarrier pairs hand each buffer on:
// vfull (TMA -> splitters), vempty (splitters -> TMA), afull (splitters -> MMA and
// epilogue: digits and row exponents written), mdone (tcgen05.commit -> splitters and
// epilogue: products complete, digit tiles free), tempty (epilogue -> MMA and splitters: TMEM
// and row exponents read).  The k-th use of a buffer waits for phase parity k & 1; a
// barrier cannot run two phases ahead of a waiter because every phase of it needs a phase the
// waiter itself completes first.  The splitters meet twice per tile at a named barrier that
// also ORs their wait failures, so they leave the loop together.  Every wait is bounded; a
// wait that runs out marks the CTA aborted, the other roles stop at their next wait, the
// epilogue writes NaN to the rows of the tiles it has not finished, and the TMA copies and MMAs
// in flight are waited for (again bounded) before TMEM is freed.
namespace {
constexpr int kPipeWarps = 18;
constexpr int kPipeThreads = kPipeWarps * 32;
constexpr int kSplitWarps = 8, kEpiWarps = 8;
constexpr int kSplitThreads = kSplitWarps * 32;
constexpr int kProdWarp = 16, kMmaWarp = 17;

struct PipeBars {
  uint64_t vfull[2], vempty[2], afull[2], mdone[2], tempty[2];
};

// Shared-memory bytes of tc_combine_pipe_kernel for padded N.
constexpr size_t pipe_smem_bytes(int NP) {
  return (size_t)2 * kDigits * kATileBytes + (size_t)kDigits * NP * kKChunk * 2 +
         (size_t)2 * kTileRows * kKChunk * 8 + sizeof(PipeBars) + 8 + 4 * kMaxN + 4 * 6 * kTileRows + 64;
}
}  // namespace

// Bounded wait for one phase of a pipeline barrier, sleeping between polls; false when the CTA
// has aborted or the polls ran out, which also marks it aborted.  The warp form gives every
// lane the same answer.
__device__ __forceinline__ bool pipe_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  bool ok = tc::mbar_wait(bar, parity, 1);   // a completed phase returns at once
  for (uint32_t r = 0; r < kPipePolls && !ok; ++r) {
    ok = tc::mbar_wait_sleep(bar, parity, 1, kPipeSleepNs);
    if (!ok && *abort_flag) break;
  }
  if (!ok) *abort_flag = 1;
  return ok;
}
__device__ __forceinline__ bool pipe_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return __all_sync(0xffffffffu, pipe_wait(bar, parity, abort_flag));
}

// Named barrier `id` over `nthreads` threads that returns the OR of every thread's `p`.
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

template <int BV, int NP>
__global__ void __launch_bounds__(kPipeThreads, 1) tc_combine_pipe_kernel(const TcArgs a) {
  constexpr uint32_t kBufCols = NP == 32 ? 256u : 128u;  // TMEM columns per buffer (7 NP used)
  constexpr size_t kBTile = (size_t)NP * kKChunk * 2;
  constexpr int kVBuf = kTileRows * kKChunk;              // doubles per V staging buffer
  constexpr int W = BV < 8 ? BV : 8;                      // columns of one block read per step
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                                        // [2][7] x 8 KB
  unsigned char* sB = sA + 2 * kDigits * kATileBytes;              // [7] x NP*64
  double* sV = reinterpret_cast<double*>(sB + kDigits * kBTile);   // [2][32 / BV][128][BV]
  PipeBars* bars = reinterpret_cast<PipeBars*>(sV + 2 * kVBuf);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  int* sF = reinterpret_cast<int*>(tslot + 2);                     // N column exponents of Y
  int* sE = sF + kMaxN;                                            // [2][128] row exponents
  int* sEp = sE + 2 * kTileRows;                                   // [4][128] unit exponents
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  {
    const int4* src = reinterpret_cast<const int4*>(a.bdig);
    int4* dst = reinterpret_cast<int4*>(sB);
    for (int e = tid; e < (int)(kDigits * kBTile / 16); e += kPipeThreads) dst[e] = src[e];
    for (int q = tid; q < a.N; q += kPipeThreads) sF[q] = a.fexp[q];
    // digit columns at or beyond K stay zero in both buffers
    int4* z = reinterpret_cast<int4*>(sA);
    for (int e = tid; e < 2 * kDigits * kATileBytes / 16; e += kPipeThreads) z[e] = make_int4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bars->vfull[b], 1);
      tc::mbar_init(&bars->vempty[b], kSplitWarps);
      tc::mbar_init(&bars->afull[b], kSplitWarps);
      tc::mbar_init(&bars->mdone[b], 1);
      tc::mbar_init(&bars->tempty[b], kEpiWarps);
    }
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (warp == kMmaWarp) {
    tc::tmem_alloc(tslot, 2 * kBufCols);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int64_t ntiles = (a.n + kTileRows - 1) / kTileRows;
  const int64_t cnt = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto tile_of = [&](int64_t it) { return (int64_t)blockIdx.x + it * gridDim.x; };
  auto bulk_ok = [&](int64_t t) {
    return a.bulk && ((uint64_t)min((int64_t)kTileRows, a.n - t * kTileRows) * BV * 8) % 16 == 0;
  };

  if (warp == kProdWarp) {
    // ---- TMA: V rows of tile `it` into staging buffer it % 2
    int64_t issued = 0;
    if (lane == 0) {
      const int nblk = a.K / BV;
      for (int64_t it = 0; it < cnt; ++it) {
        const int b = (int)(it & 1);
        const uint32_t k = (uint32_t)(it >> 1);
        if (k > 0 && !pipe_wait(&bars->vempty[b], (k - 1) & 1, abort_flag)) break;
        const int64_t r0 = tile_of(it) * kTileRows;
        if (bulk_ok(tile_of(it))) {
          const uint32_t bytes = (uint32_t)(min((int64_t)kTileRows, a.n - r0) * BV * 8);
          tc::mbar_arrive_expect_tx(&bars->vfull[b], bytes * (uint32_t)nblk);
          for (int j = 0; j < nblk; ++j)
            tc::bulk_g2s(sV + (size_t)b * kVBuf + (size_t)j * kTileRows * BV, a.vblk[j] + r0 * BV, bytes,
                         &bars->vfull[b]);
        } else {
          tc::mbar_arrive(&bars->vfull[b]);   // ragged or unaligned tile: splitters load V directly
        }
        issued = it + 1;
      }
      // copies in flight complete before the CTA exits (immediate unless the CTA aborted)
      for (int b = 0; b < 2; ++b) {
        const int64_t uses = (issued + 1 - b) / 2;
        if (uses > 0) wait_sleep(&bars->vfull[b], (uint32_t)((uses - 1) & 1));
      }
    }
  } else if (warp == kMmaWarp) {
    // ---- MMA issue: digit i of A against the B digit tiles 0..6-i stacked as one (7-i) NP-row
    // operand; the product's column block j lands on class i + j's accumulator (TMEM column
    // (i + j) NP of buffer it % 2)
    int64_t committed = 0;
    if (lane == 0) {
      const int ksteps = a.K <= 16 ? 1 : 2;   // K-steps of 16 holding non-zero digits
      const uint32_t sa0 = tc::smem_addr(sA), sb0 = tc::smem_addr(sB);
      const uint64_t bd = tc::smem_desc(sb0, kLBO, kSBO);
      for (int64_t it = 0; it < cnt; ++it) {
        const int b = (int)(it & 1);
        const uint32_t k = (uint32_t)(it >> 1);
        if (!pipe_wait(&bars->afull[b], k & 1, abort_flag)) break;
        if (k > 0 && !pipe_wait(&bars->tempty[b], (k - 1) & 1, abort_flag)) break;
        tc::fence_after_sync();
        const uint32_t dbase = tbase + (uint32_t)b * kBufCols;
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
          const uint64_t ad = tc::smem_desc(sa0 + (uint32_t)((b * kDigits + i) * kATileBytes), kLBO, kSBO);
          const uint32_t idesc = tc::idesc_f16_f32(kTileRows, (kDigits - i) * NP);
          for (int ks = 0; ks < ksteps; ++ks)
            tc::mma_f16(dbase + (uint32_t)(i * NP), ad + (uint64_t)(ks * 2 * kLBO >> 4),
                        bd + (uint64_t)(ks * 2 * kLBO >> 4), idesc, (i > 0 || ks > 0) ? 1u : 0u);
        }
        tc::mma_commit(&bars->mdone[b]);
        committed = it + 1;
      }
      for (int b = 0; b < 2; ++b) {
        const int64_t uses = (committed + 1 - b) / 2;
        if (uses > 0) wait_sleep(&bars->mdone[b], (uint32_t)((uses - 1) & 1));
      }
    }
  } else if (warp < kSplitWarps) {
    // ---- split: units of 8 columns of one row
    const int nunits = kTileRows * ((a.K + 7) >> 3);
    for (int64_t it = 0; it < cnt; ++it) {
      const int b = (int)(it & 1);
      const uint32_t k = (uint32_t)(it >> 1);
      const int64_t tile = tile_of(it);
      const bool bulk = bulk_ok(tile);
      const bool ok = pipe_wait_warp(&bars->vfull[b], k & 1, abort_flag);
      double v[2][8];
      int emax[2] = {0, 0};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int u = tid + kSplitThreads * j;
        if (u < nunits) {
          const int row = u & (kTileRows - 1), cb = u >> 7;
          const int64_t r = tile * kTileRows + row;
          const bool live = r < a.n;
#pragma unroll
          for (int c0 = 0; c0 < 8; c0 += W) {
            const int c = cb * 8 + c0;
            if (live && c < a.K) {
              const double* src = bulk ? sV + (size_t)b * kVBuf + ((size_t)(c / BV) * kTileRows + row) * BV + c % BV
                                       : a.vblk[c / BV] + r * BV + c % BV;
              if (bulk && W % 2 == 0) {
#pragma unroll
                for (int p = 0; p < W; p += 2) {
                  const double2 x = *reinterpret_cast<const double2*>(src + p);
                  v[j][c0 + p] = x.x;
                  v[j][c0 + p + 1] = x.y;
                }
              } else {
#pragma unroll
                for (int p = 0; p < W; ++p) v[j][c0 + p] = src[p];
              }
            } else {
#pragma unroll
              for (int p = 0; p < W; ++p) v[j][c0 + p] = 0.0;
            }
          }
          int e = 0;
#pragma unroll
          for (int c = 0; c < 8; ++c) e = max(e, exp_field(v[j][c]));
          sEp[cb * kTileRows + row] = e;
        }
      }
      if (bar_or(1, kSplitThreads, !ok)) break;   // V read, unit exponents written
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->vempty[b]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int u = tid + kSplitThreads * j;
        if (u < nunits) {
          const int row = u & (kTileRows - 1);
          for (int c = 0; c < nunits / kTileRows; ++c) emax[j] = max(emax[j], sEp[c * kTileRows + row]);
        }
      }
      // digit tiles and row exponents of this buffer are free once tile it - 2's products and
      // results are done
      bool ok2 = true;
      if (k > 0) ok2 = pipe_wait_warp(&bars->mdone[b], (k - 1) & 1, abort_flag) &&
                       pipe_wait_warp(&bars->tempty[b], (k - 1) & 1, abort_flag);
      if (bar_or(1, kSplitThreads, !ok2)) break;  // unit exponents read
      unsigned char* sAb = sA + (size_t)b * kDigits * kATileBytes;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int u = tid + kSplitThreads * j;
        if (u < nunits) {
          const int row = u & (kTileRows - 1), cb = u >> 7;
          if (cb == 0) sE[b * kTileRows + row] = emax[j];
          uint32_t w[kDigits][4];
          split_pair_f16(v[j][0], v[j][1], emax[j], w, 0);
          split_pair_f16(v[j][2], v[j][3], emax[j], w, 1);
          split_pair_f16(v[j][4], v[j][5], emax[j], w, 2);
          split_pair_f16(v[j][6], v[j][7], emax[j], w, 3);
          const uint32_t off = tile_off(row, cb * 8);
#pragma unroll
          for (int i = 0; i < kDigits; ++i)
            *reinterpret_cast<uint4*>(sAb + (size_t)i * kATileBytes + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
        }
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->afull[b]);
    }
  } else {
    // ---- epilogue: warps 8-15, TMEM lane quarter warp % 4; the two warps of a quarter take
    // alternate groups of two results (q0 = 2 half + 4 jj)
    const int quarter = warp & 3, half = (warp - kSplitWarps) >> 2;
    const int row = quarter * 32 + lane;
    const bool add_out = a.beta != 0.0;
    const int ngroups = (a.N - 2 * half + 3) / 4;        // this thread's groups of two results
    // rows of Out loaded ahead of their tile: one group per thread (N <= 4) two tiles ahead into
    // slot it % 2, two groups (N <= 8) one tile ahead into slot = group
    const int pf = !add_out ? 0 : ngroups <= 1 ? 2 : ngroups == 2 ? 1 : 0;
    double opf[2][2];
    auto load_grp = [&](int64_t it, int jj, int slot) {
      const int64_t r = tile_of(it) * kTileRows + row;
      const int q0 = 2 * half + 4 * jj;
      if (r >= a.n || q0 >= a.N) return;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = q0 + u;
        const double x = q < a.N ? a.oblk[q / BV][r * BV + q % BV] : 0.0;
        if (slot == 0) opf[0][u] = x;
        else opf[1][u] = x;
      }
    };
    if (pf == 2) {
      if (cnt > 0) load_grp(0, 0, 0);
      if (cnt > 1) load_grp(1, 0, 1);
    } else if (pf == 1 && cnt > 0) {
      load_grp(0, 0, 0);
      load_grp(0, 1, 1);
    }
    int64_t it = 0;
    for (; it < cnt; ++it) {
      const int b = (int)(it & 1);
      const uint32_t k = (uint32_t)(it >> 1);
      if (!pipe_wait_warp(&bars->afull[b], k & 1, abort_flag)) break;
      if (!pipe_wait_warp(&bars->mdone[b], k & 1, abort_flag)) break;
      tc::fence_after_sync();
      const int64_t r = tile_of(it) * kTileRows + row;
      const bool live = r < a.n;
      const int emax = sE[b * kTileRows + row];
      const int ebase = emax - 2108 + kAsmShift;
      const uint32_t lane_addr = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * kBufCols;
      // the accumulators of group jj + 1 are loaded while group jj is assembled
      uint32_t nxt[kClasses][2];
      if (ngroups > 0) {
#pragma unroll
        for (int g = 0; g < kClasses; ++g) tc::tmem_ld2(lane_addr + (uint32_t)(g * NP + 2 * half), nxt[g]);
      }
      for (int jj = 0; jj < ngroups; ++jj) {
        const int q0 = 2 * half + 4 * jj;
        tc::tmem_ld_wait();
        uint32_t acc[kClasses][2];
#pragma unroll
        for (int g = 0; g < kClasses; ++g) {
          tc::reg_after_wait(nxt[g]);
          acc[g][0] = nxt[g][0];
          acc[g][1] = nxt[g][1];
        }
        if (jj + 1 < ngroups) {
#pragma unroll
          for (int g = 0; g < kClasses; ++g) tc::tmem_ld2(lane_addr + (uint32_t)(g * NP + q0 + 4), nxt[g]);
        }
        if (jj == ngroups - 1) {
          // TMEM buffer and row exponent read: the buffer goes back to the MMA issuer
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&bars->tempty[b]);
        }
        double y[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int64_t hi = (int64_t)acc_int(acc[0][u]) * 65536 + (int64_t)acc_int(acc[1][u]) * 256 +
                             (int64_t)acc_int(acc[2][u]);
          const int64_t lo = (int64_t)acc_int(acc[3][u]) * 16777216 + (int64_t)acc_int(acc[4][u]) * 65536 +
                             (int64_t)acc_int(acc[5][u]) * 256 + (int64_t)acc_int(acc[6][u]);
          const double x = assemble(hi, lo, ebase + sF[min(q0 + u, kMaxN - 1)]);
          y[u] = emax > 0 ? x : 0.0;
        }
        if (live) {
          if (add_out) {
            if (pf != 0) {
              const bool s1 = pf == 2 ? (it & 1) != 0 : jj != 0;
#pragma unroll
              for (int u = 0; u < 2; ++u) y[u] = fma(a.beta, s1 ? opf[1][u] : opf[0][u], y[u]);
            } else {
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int q = q0 + u;
                if (q < a.N) y[u] = fma(a.beta, a.oblk[q / BV][r * BV + q % BV], y[u]);
              }
            }
          }
          if (BV >= 2 && q0 + 2 <= a.N && a.ovec) {
            *reinterpret_cast<double2*>(a.oblk[q0 / BV] + r * BV + q0 % BV) = make_double2(y[0], y[1]);
          } else {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int q = q0 + u;
              if (q < a.N) a.oblk[q / BV][r * BV + q % BV] = y[u];
            }
          }
        }
      }
      if (ngroups == 0) {
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bars->tempty[b]);
      }
      if (pf == 2 && it + 2 < cnt) load_grp(it + 2, 0, (int)(it & 1));
      if (pf == 1 && it + 1 < cnt) {
        load_grp(it + 1, 0, 0);
        load_grp(it + 1, 1, 1);
      }
    }
    // after an abort: the rows of every tile not finished read NaN
    for (; it < cnt; ++it) {
      const int64_t r = tile_of(it) * kTileRows + row;
      if (r < a.n)
        for (int jj = 0; jj < ngroups; ++jj)
          for (int q = 2 * half + 4 * jj; q < min(a.N, 2 * half + 4 * jj + 2); ++q)
            a.oblk[q / BV][r * BV + q % BV] = __longlong_as_double(0x7FF8000000000000ll);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0 && *abort_flag) atomicExch(a.status, 1);
  if (warp == kMmaWarp) tc::tmem_dealloc(tbase, 2 * kBufCols);
}

template <int BV, int NP>
static int launch_tc_combine_pipe_np(const TcArgs& a, cudaStream_t s) {
  static KernelSetup ks;
  const void* fn = reinterpret_cast<const void*>(tc_combine_pipe_kernel<BV, NP>);
  constexpr size_t smem = pipe_smem_bytes(NP);
  FE_TRY(kernel_configure(ks, fn, (int)smem));
  const int64_t ntiles = ceil_div(a.n, kTileRows);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms()));
  tc_combine_pipe_kernel<BV, NP><<<(unsigned)grid, kPipeThreads, smem, s>>>(a);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

template <int BV>
static int launch_tc_combine_pipe(const TcArgs& a, cudaStream_t s) {
  if (a.NP == 16) return launch_tc_combine_pipe_np<BV, 16>(a, s);
  return launch_tc_combine_pipe_np<BV, 32>(a, s);
}

bool tc_combine_supported(const BlockSet& V, const BlockSet& Out, fe_dtype dt) {
  const int K = V.nv * V.bv, N = Out.nv * Out.bv;
  return dt == FE_F64 && V.bv == Out.bv && V.ld == V.bv && Out.ld == Out.bv && K >= 1 && K <= kMaxK &&
         N >= 1 && N <= kMaxN && V.bv >= 1 && V.bv <= 16;
}

template <int BV, int KMAX>
static int launch_tc_combine(const TcArgs& a, size_t smem, bool two_per_sm, cudaStream_t s) {
  static KernelSetup ks;
  const void* fn = reinterpret_cast<const void*>(tc_combine_kernel<BV, KMAX>);
  FE_TRY(kernel_configure(ks, fn, 227 * 1024));
  const int64_t ntiles = ceil_div(a.n, kTileRows);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)(two_per_sm ? 2 : 1) * num_sms()));
  tc_combine_kernel<BV, KMAX><<<(unsigned)grid, kThreads, smem, s>>>(a);
  count_launch();
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

template <int BV>
static int launch_tc_combine_k(const TcArgs& a, size_t smem, bool two_per_sm, cudaStream_t s) {
  if (a.K <= 32) return launch_tc_combine<BV, 32>(a, smem, two_per_sm, s);
  return launch_tc_combine<BV, 64>(a, smem, two_per_sm, s);
}

// Out = V Y on the tensor cores (FP64 blocks; see tc_combine_supported for the shapes).
int tc_combine(const BlockSet& V, int64_t n, const double* Y, int ldy, const BlockSet& Out,
               cudaStream_t s, double alpha, double beta) {
  FE_ARG(tc_combine_supported(V, Out, FE_F64), "tc_combine: unsupported shape");
  TcArgs a;
  memset(&a, 0, sizeof(a));
  const int BV = V.bv;
  a.n = n;
  a.K = V.nv * BV;
  a.N = Out.nv * BV;
  a.NP = a.N <= 16 ? 16 : 32;
  a.nkc = (int)ceil_div(a.K, kKChunk);
  a.beta = beta;
  a.bulk = 1;
  for (int j = 0; j < V.nv; ++j) {
    a.vblk[j] = static_cast<const double*>(V.blk[j]);
    if (reinterpret_cast<uintptr_t>(V.blk[j]) % 16) a.bulk = 0;
  }
  a.ovec = 1;
  for (int o = 0; o < Out.nv; ++o) {
    a.oblk[o] = const_cast<double*>(static_cast<const double*>(Out.blk[o]));
    if (reinterpret_cast<uintptr_t>(Out.blk[o]) % 16) a.ovec = 0;
  }
  // scratch: B digit tiles, column exponents, status word
  const size_t bbytes = (size_t)a.nkc * kDigits * a.NP * kKChunk * 2;
  double* scr = small_scratch(17, bbytes / 8 + kMaxN + 2);
  if (!scr) return FE_ERR_OOM;
  a.bdig = reinterpret_cast<const uint16_t*>(scr);
  a.fexp = reinterpret_cast<const int*>(scr + bbytes / 8);
  a.status = reinterpret_cast<int*>(scr + bbytes / 8 + kMaxN);
  FE_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), s));
  tc_prep_y_kernel<<<1, 256, 0, s>>>(Y, ldy, alpha, a.K, a.N, a.NP, a.nkc, const_cast<uint16_t*>(a.bdig),
                                     const_cast<int*>(a.fexp));
  count_launch();
  FE_CUDA(cudaGetLastError());
  if (a.nkc == 1) {
    switch (BV) {
      case 1: return launch_tc_combine_pipe<1>(a, s);
      case 2: return launch_tc_combine_pipe<2>(a, s);
      case 4: return launch_tc_combine_pipe<4>(a, s);
      case 8: return launch_tc_combine_pipe<8>(a, s);
      case 16: return launch_tc_combine_pipe<16>(a, s);
    }
  }
  // two CTAs per SM when their TMEM (256 columns each) fits; the shared-memory request keeps a
  // third CTA off the SM, so no CTA waits in tcgen05.alloc
  const bool two = a.nkc * kClasses * a.NP <= 256;
  const size_t smem = std::max(tc_smem_bytes(a.nkc, a.NP), two ? (size_t)100 * 1024 : (size_t)120 * 1024);
  switch (BV) {
    case 1: return launch_tc_combine_k<1>(a, smem, two, s);
    case 2: return launch_tc_combine_k<2>(a, smem, two, s);
    case 4: return launch_tc_combine_k<4>(a, smem, two, s);
    case 8: return launch_tc_combine_k<8>(a, smem, two, s);
    case 16: return launch_tc_combine_k<16>(a, smem, two, s);
  }
  return set_error(FE_ERR_INVALID, "tc_combine: block width %d", BV);
}


// ---------------------------------------------------------------- Gram V^T W (op3)
// G = alpha V^T W for FP64 blocks on the tensor cores (Table 1 "op3", MvTransMv), the same
// digit splitting as above with the roles of rows and columns exchanged: the contraction runs
// over the rows, so every column of V and of W is scaled by its largest exponent within each
// 128-row tile.  Per tile the MMA multiplies ALL digit slices at once: A holds the digit rows
// (i, c) of V^T (7 * KV <= 252 rows, two 128-row M tiles), B the digit rows (j, q) of W^T
// (7 * bw rows), K = the tile's 128 rows; every accumulator D[(i, c)][(j, q)] sums 128
// products below 2^16 and is exact.  TMEM lane (i, c) then forms T_i = sum_j D 2^(8 (6 - j))
// for each q in 64-bit integers; the seven slices i of each output are added exactly in
// 128-bit integers, and the sum, scaled by the tile's column exponents, is rounded once to FP64
// and added to the CTA's accumulator of G, and the CTAs' partial Gram matrices are added in a fixed order.
// Error per tile: 2^-50 * 128 * max|V[., c]| * max|W[., q]| over the tile's rows, plus the FP64
// roundings of the sums over tiles and CTAs.
namespace {
constexpr int kGramMaxKV = 36;                       // 7 * 36 = 252 digit rows of V^T
constexpr int kGramMaxBW = 8;                        // 7 * 8 = 56 digit rows of W^T
constexpr int kGramRows = 128;                       // rows per tile (MMA K = 8 x 16)
constexpr uint32_t kGSBO = (kGramRows / 8) * kCoreBytes;  // 2048 B between 8-row groups
constexpr int kGATile = 128 * kGramRows * 2;         // one 128-row M tile of V^T digits: 32 KB

struct TcGramArgs {
  const double* vblk[kMaxBlocks];
  int bv, KV;            // V: KV / bv blocks of n x bv (ld bv)
  const double* W;
  int bw, NP;            // W: n x bw (ld bw); NP = 7 bw padded to the MMA's N
  int nmt;               // M tiles of V^T digits (1 or 2)
  int64_t n;
  double* partial;       // [gridDim.x][KV * bw]
  int* status;
  int bulk;              // 1: V blocks and W 16-byte aligned (TMA bulk copies allowed)
  int nxb;               // staging buffers of the pipelined kernel (1 or 2)
};
}  // namespace

// ---------------------------------------------------------------- pipelined Gram
// The same Gram with its phases overlapped, in the warp roles of the pipelined block product:
//   warps 0-11  split: unit u = 16 c + g (column c of [V W], 8-row group g), thread t takes
//               units t and t + 384; the 16 lanes of a half-warp hold one column, so its
//               exponent over the tile is a 4-step shuffle maximum; digits go to the A / B tiles
//               of buffer t % 2;
//   warp 16     (one thread) TMA copies of the tile's rows into the (single) staging buffer;
//   warp 17     (one thread) the nmt x 8 MMAs of a tile into TMEM buffer t % 2;
//   warps 12-15 (TMEM lane quarter = warp % 4) for every lane (i, c) and column q:
//               T_i = sum_j D[(i,c)][(j,q)] 2^(8 (6 - j)) as an integer (the 12 low bits
//               dropped), into shared memory; after a barrier of the four warps, each output
//               (c, q) sums its seven slices exactly in 128-bit integers, sum_i T_i 2^(8 (6 - i)),
//               converts once (truncation) to FP64 with the tile's column scales and adds it to
//               the thread's FP64 partial of G.
// Barriers: xfull / xempty (staging), afull / mdone / tempty per buffer, as in the block
// product; the splitters meet twice per tile and the epilogue warps twice, at named barriers
// that OR their wait failures.
namespace {
constexpr int kGSplitWarps = 12, kGEpiWarps = 4;
constexpr int kGSplitThreads = kGSplitWarps * 32;
constexpr int kGEpiThreads = kGEpiWarps * 32;
constexpr int kGProdWarp = 16, kGMmaWarp = 17;
constexpr int kGPipeThreads = 18 * 32;

struct GramBars {
  uint64_t xfull[2], xempty[2], afull[2], mdone[2], tempty[2];
};
constexpr int kGramMaxCols = kGramMaxKV + kGramMaxBW;

struct GramPipeLayout {
  size_t a, b, x, xbuf, t, e, bars, total;
  int nxb;   // staging buffers: 2 when they fit, else 1
};
__host__ __device__ inline GramPipeLayout gram_pipe_layout(int nmt, int NP, int nvb, int bv, int bw, int KV,
                                                          int nxb) {
  GramPipeLayout L;
  L.nxb = nxb;
  L.a = 0;
  L.b = L.a + (size_t)2 * nmt * kGATile;
  L.x = L.b + (size_t)2 * NP * kGramRows * 2;
  const size_t xd = (size_t)nvb * (kGramRows * bv + 4) + (size_t)kGramRows * bw + 4;
  L.xbuf = (xd * 8 + 15) & ~(size_t)15;
  L.t = L.x + (size_t)nxb * L.xbuf;
  L.e = L.t + (size_t)7 * KV * bw * 8;
  L.bars = (L.e + (size_t)4 * kGramMaxCols * 4 + 15) & ~(size_t)15;
  L.total = L.bars + sizeof(GramBars) + 16;
  return L;
}

// |v| < 2^127 times 2^s, truncated to FP64 (zero below the normal range, infinity above it).
__device__ __forceinline__ double i128_to_double(__int128 v, int s) {
  const uint64_t sign = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned __int128 a = v < 0 ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
  const uint32_t w3 = (uint32_t)(hi >> 32), w2 = (uint32_t)hi, w1 = (uint32_t)(lo >> 32), w0 = (uint32_t)lo;
  const int lz = w3 != 0 ? __clz(w3) : w2 != 0 ? 32 + __clz(w2) : w1 != 0 ? 64 + __clz(w1) : 96 + __clz(w0);
  const unsigned __int128 nrm = a << (lz & 127);
  const uint64_t m = (uint64_t)(nrm >> 64);
  const int ef = 127 - lz + s + 1023;
  uint64_t bits = sign | ((uint64_t)(uint32_t)ef << 52) | ((m >> 11) & 0xFFFFFFFFFFFFFull);
  bits = (a == 0 || ef <= 0) ? sign : bits;
  bits = ef >= 2047 ? (sign | 0x7FF0000000000000ull) : bits;
  return __longlong_as_double((long long)bits);
}
}  // namespace

template <int BW>
__global__ void __launch_bounds__(kGPipeThreads, 1) tc_gram_pipe_kernel(const TcGramArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int bw = BW;
  constexpr int NP = (7 * BW + 15) / 16 * 16;
  const int KV = a.KV, nmt = a.nmt, bv = a.bv;
  const int ncol = KV + bw;
  const int nvb = KV / bv;
  const int XS = kGramRows * bv + 4;           // doubles per staged V block (padded)
  const GramPipeLayout L = gram_pipe_layout(nmt, NP, nvb, bv, bw, KV, a.nxb);
  const int nxb = a.nxb;
  unsigned char* sA = smem + L.a;              // [2][nmt] x 32 KB
  unsigned char* sB = smem + L.b;              // [2] x NP x 128 FP16
  double* sX = reinterpret_cast<double*>(smem + L.x);
  int64_t* sT = reinterpret_cast<int64_t*>(smem + L.t);   // [bw][7][KV] slice integers
  int* sEx = reinterpret_cast<int*>(smem + L.e);          // [2][ncol] column exponents by buffer
  int* sExw = sEx + 2 * kGramMaxCols;                      // [2][ncol] maxima being formed
  GramBars* bars = reinterpret_cast<GramBars*>(smem + L.bars);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bufcols = nmt * NP <= 64 ? 64u : 128u;

  {
    int4* z = reinterpret_cast<int4*>(smem);
    for (int e = tid; e < (int)(L.x / 16); e += kGPipeThreads) z[e] = make_int4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bars->xfull[b], 1);
      tc::mbar_init(&bars->xempty[b], kGSplitWarps);
      tc::mbar_init(&bars->afull[b], kGSplitWarps);
      tc::mbar_init(&bars->mdone[b], 1);
      tc::mbar_init(&bars->tempty[b], kGEpiWarps);
    }
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (warp == kGMmaWarp) {
    tc::tmem_alloc(tslot, 2 * bufcols);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int64_t ntiles = (a.n + kGramRows - 1) / kGramRows;
  const int64_t cnt = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto tile_of = [&](int64_t it) { return (int64_t)blockIdx.x + it * gridDim.x; };
  auto bulk_ok = [&](int64_t t) {
    const int64_t rows = min((int64_t)kGramRows, a.n - t * kGramRows);
    return a.bulk && (rows * bv * 8) % 16 == 0 && (rows * bw * 8) % 16 == 0;
  };

  if (warp == kGProdWarp) {
    int64_t issued = 0;
    if (lane == 0) {
      for (int64_t it = 0; it < cnt; ++it) {
        const int xb = nxb == 2 ? (int)(it & 1) : 0;
        const int64_t xk = nxb == 2 ? (it >> 1) : it;
        if (xk > 0 && !pipe_wait(&bars->xempty[xb], (uint32_t)((xk - 1) & 1), abort_flag)) break;
        const int64_t t = tile_of(it), r0 = t * kGramRows;
        double* sXb = sX + (size_t)xb * (L.xbuf / 8);
        if (bulk_ok(t)) {
          const int64_t rows = min((int64_t)kGramRows, a.n - r0);
          const uint32_t vb = (uint32_t)(rows * bv * 8), wb = (uint32_t)(rows * bw * 8);
          tc::mbar_arrive_expect_tx(&bars->xfull[xb], vb * (uint32_t)nvb + wb);
          for (int j = 0; j < nvb; ++j) tc::bulk_g2s(sXb + (size_t)j * XS, a.vblk[j] + r0 * bv, vb, &bars->xfull[xb]);
          tc::bulk_g2s(sXb + (size_t)nvb * XS, a.W + r0 * bw, wb, &bars->xfull[xb]);
        } else {
          tc::mbar_arrive(&bars->xfull[xb]);   // ragged or unaligned tile: splitters load directly
        }
        issued = it + 1;
      }
      for (int xb = 0; xb < nxb; ++xb) {
        const int64_t uses = nxb == 2 ? (issued + 1 - xb) / 2 : issued;
        if (uses > 0) wait_sleep(&bars->xfull[xb], (uint32_t)((uses - 1) & 1));
      }
    }
  } else if (warp == kGMmaWarp) {
    int64_t committed = 0;
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16_f32(128, NP);
      const uint32_t sa0 = tc::smem_addr(sA), sb0 = tc::smem_addr(sB);
      for (int64_t it = 0; it < cnt; ++it) {
        const int b = (int)(it & 1);
        const uint32_t k = (uint32_t)(it >> 1);
        if (!pipe_wait(&bars->afull[b], k & 1, abort_flag)) break;
        if (k > 0 && !pipe_wait(&bars->tempty[b], (k - 1) & 1, abort_flag)) break;
        tc::fence_after_sync();
        for (int mt = 0; mt < nmt; ++mt)
#pragma unroll
          for (int ks = 0; ks < kGramRows / 16; ++ks) {
            const uint64_t ad = tc::smem_desc(sa0 + (uint32_t)((b * nmt + mt) * kGATile + ks * 2 * kCoreBytes),
                                              kCoreBytes, kGSBO);
            const uint64_t bd = tc::smem_desc(sb0 + (uint32_t)(b * NP * kGramRows * 2 + ks * 2 * kCoreBytes),
                                              kCoreBytes, kGSBO);
            tc::mma_f16(tbase + (uint32_t)b * bufcols + (uint32_t)(mt * NP), ad, bd, idesc, ks > 0 ? 1u : 0u);
          }
        tc::mma_commit(&bars->mdone[b]);
        committed = it + 1;
      }
      for (int b = 0; b < 2; ++b) {
        const int64_t uses = (committed + 1 - b) / 2;
        if (uses > 0) wait_sleep(&bars->mdone[b], (uint32_t)((uses - 1) & 1));
      }
    }
  } else if (warp < kGSplitWarps) {
    // ---- split: units (column c, 8-row group g) with u = g ncol + c, so that a warp's lanes read
    // and write neighbouring columns (no shared-memory bank conflicts); the column exponents
    // are maxima over the 16 groups through shared-memory atomics (double-buffered by tile)
    const int nunits = ncol * 16;
    // this thread's units, the same in every tile: column, row group, column pointer and stride
    int uc[2], ug[2], ustr[2], usoff[2];
    const double* ucol[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int u = tid + kGSplitThreads * j;
      uc[j] = u < nunits ? u % ncol : 0;
      ug[j] = u < nunits ? u / ncol : 0;
      const int c = uc[j];
      const bool isv = c < KV;
      ustr[j] = isv ? bv : bw;
      ucol[j] = isv ? a.vblk[c / bv] + c % bv : a.W + (c - KV);
      usoff[j] = isv ? (c / bv) * XS + c % bv : nvb * XS + (c - KV);
    }
    for (int e = tid; e < 2 * kGramMaxCols; e += kGSplitThreads) sExw[e] = 0;
    bar_or(1, kGSplitThreads, false);
    for (int64_t it = 0; it < cnt; ++it) {
      const int b = (int)(it & 1);
      const uint32_t k = (uint32_t)(it >> 1);
      const int64_t t = tile_of(it), r0 = t * kGramRows;
      const bool bulk = bulk_ok(t);
      int* exw = sExw + (it & 1) * kGramMaxCols;
      const int xb = nxb == 2 ? (int)(it & 1) : 0;
      const double* sXb = sX + (size_t)xb * (L.xbuf / 8);
      const bool ok = pipe_wait_warp(&bars->xfull[xb], (uint32_t)((nxb == 2 ? (it >> 1) : it) & 1), abort_flag);
      double x[2][8];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int u = tid + kGSplitThreads * j;
        if (u < nunits) {
          const int c = uc[j], g = ug[j], str = ustr[j];
          const double* gcol = ucol[j];
          const double* scol = sXb + usoff[j];
          int e = 0;
          if (bulk) {
#pragma unroll
            for (int tt = 0; tt < 8; ++tt) {
              const double v = scol[(g * 8 + tt) * str];   // in the staging buffer in any case
              x[j][tt] = r0 + g * 8 + tt < a.n ? v : 0.0;
            }
          } else {
#pragma unroll
            for (int tt = 0; tt < 8; ++tt) {
              const int64_t r = r0 + g * 8 + tt;
              x[j][tt] = r < a.n ? __ldg(gcol + r * str) : 0.0;
            }
          }
#pragma unroll
          for (int tt = 0; tt < 8; ++tt) e = max(e, exp_field(x[j][tt]));
          if (e > 0) atomicMax(exw + c, e);
        }
      }
      if (bar_or(1, kGSplitThreads, !ok)) break;   // staging buffer read, exponent maxima formed
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->xempty[xb]);
      int emax[2] = {0, 0};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int u = tid + kGSplitThreads * j;
        if (u < nunits) emax[j] = exw[uc[j]];
      }
      // the other buffer of maxima (read by everyone before the previous tile's second barrier)
      // starts the next tile at zero
      for (int e = tid; e < ncol; e += kGSplitThreads) sExw[((it + 1) & 1) * kGramMaxCols + e] = 0;
      bool ok2 = true;
      if (k > 0) ok2 = pipe_wait_warp(&bars->mdone[b], (k - 1) & 1, abort_flag) &&
                       pipe_wait_warp(&bars->tempty[b], (k - 1) & 1, abort_flag);
      if (bar_or(1, kGSplitThreads, !ok2)) break;  // digit tiles and exponents of buffer b free
      unsigned char* sAb = sA + (size_t)b * nmt * kGATile;
      unsigned char* sBb = sB + (size_t)b * NP * kGramRows * 2;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int u = tid + kGSplitThreads * j;
        if (u < nunits) {
          const int c = uc[j], g = ug[j];
          if (g == 0) sEx[b * kGramMaxCols + c] = emax[j];
          uint32_t w[kDigits][4];
          split_pair_f16(x[j][0], x[j][1], emax[j], w, 0);
          split_pair_f16(x[j][2], x[j][3], emax[j], w, 1);
          split_pair_f16(x[j][4], x[j][5], emax[j], w, 2);
          split_pair_f16(x[j][6], x[j][7], emax[j], w, 3);
#pragma unroll
          for (int i = 0; i < kDigits; ++i) {
            unsigned char* dst;
            if (c < KV) {
              const int m = i * KV + c;
              dst = sAb + (size_t)(m >> 7) * kGATile + ((m & 127) >> 3) * kGSBO + g * kCoreBytes + (m & 7) * 16;
            } else {
              const int nn = i * bw + (c - KV);
              dst = sBb + (nn >> 3) * kGSBO + g * kCoreBytes + (nn & 7) * 16;
            }
            *reinterpret_cast<uint4*>(dst) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
          }
        }
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->afull[b]);
    }
  } else if (warp < kGSplitWarps + kGEpiWarps) {
    // ---- epilogue: TMEM lane quarter warp % 4 of each M tile
    const int quarter = warp & 3, et = tid - kGSplitThreads;
    const int nout = KV * bw;
    double acc[3] = {0.0, 0.0, 0.0};   // outputs et, et + 128, et + 256 (nout <= 288)
    for (int64_t it = 0; it < cnt; ++it) {
      const int b = (int)(it & 1);
      const uint32_t k = (uint32_t)(it >> 1);
      const bool ok = pipe_wait_warp(&bars->afull[b], k & 1, abort_flag) &&
                      pipe_wait_warp(&bars->mdone[b], k & 1, abort_flag);
      if (bar_or(2, kGEpiThreads, !ok)) break;
      tc::fence_after_sync();
      // this thread's output scales, read before the buffer's exponents are handed back
      const int* ex = sEx + b * kGramMaxCols;
      int scl[3];
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        const int o = et + kGEpiThreads * kk;
        scl[kk] = 0;
        if (o < nout) {
          const int ec = ex[o / bw], fq = ex[KV + o % bw];
          scl[kk] = ec > 0 && fq > 0 ? ec + fq : 0;
        }
      }
      for (int mt = 0; mt < nmt; ++mt) {
        const int m = mt * 128 + quarter * 32 + lane;
        const uint32_t laddr = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * bufcols + (uint32_t)(mt * NP);
#pragma unroll
        for (int q = 0; q < bw; ++q) {
          uint32_t d[kDigits];
#pragma unroll
          for (int jd = 0; jd < kDigits; ++jd) d[jd] = tc::tmem_ld1(laddr + (uint32_t)(jd * bw + q));
          tc::tmem_ld_wait();
#pragma unroll
          for (int jd = 0; jd < kDigits; ++jd) tc::reg_after_wait(d[jd]);
          if (m < 7 * KV) {
            const int64_t hi = (int64_t)acc_int(d[0]) * 65536 + (int64_t)acc_int(d[1]) * 256 + (int64_t)acc_int(d[2]);
            const int64_t lo = (int64_t)acc_int(d[3]) * 16777216 + (int64_t)acc_int(d[4]) * 65536 +
                               (int64_t)acc_int(d[5]) * 256 + (int64_t)acc_int(d[6]);
            // T_i / 2^12 (floor), i = m / KV, c = m % KV
            sT[q * 7 * KV + m] = (hi << (32 - kAsmShift)) + (lo >> kAsmShift);
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->tempty[b]);
      bar_or(2, kGEpiThreads, false);   // slice integers written
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        const int o = et + kGEpiThreads * kk;
        if (o < nout) {
          const int c = o / bw, q = o % bw;
          __int128 sum = 0;
#pragma unroll
          for (int i = 0; i < kDigits; ++i) sum += (__int128)sT[q * 7 * KV + i * KV + c] << (8 * (6 - i));
          if (scl[kk] > 0) acc[kk] += i128_to_double(sum, scl[kk] - 2108 + kAsmShift - 48);
        }
      }
      bar_or(2, kGEpiThreads, false);   // slice integers read: the next tile may overwrite them
    }
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const int o = et + kGEpiThreads * kk;
      if (o < nout) a.partial[(int64_t)blockIdx.x * nout + o] = *abort_flag ? __longlong_as_double(0x7FF8000000000000ll) : acc[kk];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0 && *abort_flag) atomicExch(a.status, 1);
  if (warp == kGMmaWarp) tc::tmem_dealloc(tbase, 2 * bufcols);
}

bool tc_gram_supported(const BlockSet& V, int bw, int ldw, fe_dtype dt) {
  const int KV = V.nv * V.bv;
  return dt == FE_F64 && V.ld == V.bv && ldw == bw && KV >= 1 && KV <= kGramMaxKV &&
         (bw == 1 || bw == 2 || bw == 4 || bw == 8) && V.bv >= 1;
}

int tc_gram(const BlockSet& V, int64_t n, const double* W, int bw, double alpha, double* G,
            cudaStream_t s) {
  FE_ARG(tc_gram_supported(V, bw, bw, FE_F64), "tc_gram: unsupported shape");
  TcGramArgs a;
  memset(&a, 0, sizeof(a));
  a.bv = V.bv;
  a.KV = V.nv * V.bv;
  for (int j = 0; j < V.nv; ++j) a.vblk[j] = static_cast<const double*>(V.blk[j]);
  a.W = W;
  a.bw = bw;
  a.bulk = reinterpret_cast<uintptr_t>(W) % 16 == 0;
  for (int j = 0; j < V.nv; ++j)
    if (reinterpret_cast<uintptr_t>(V.blk[j]) % 16) a.bulk = 0;
  a.NP = (int)ceil_div(7 * bw, 16) * 16;
  a.nmt = (int)ceil_div(7 * a.KV, 128);
  a.n = n;
  GramPipeLayout L = gram_pipe_layout(a.nmt, a.NP, a.KV / a.bv, a.bv, bw, a.KV, 2);
  if (L.total > 227 * 1024) L = gram_pipe_layout(a.nmt, a.NP, a.KV / a.bv, a.bv, bw, a.KV, 1);
  a.nxb = L.nxb;
  FE_ARG(L.total <= 227 * 1024 && a.KV * bw <= 3 * kGEpiThreads, "tc_gram: shape too large");
  static KernelSetup kp[4];
  const int bj = bw == 1 ? 0 : bw == 2 ? 1 : bw == 4 ? 2 : 3;
  const void* fp = bw == 1 ? reinterpret_cast<const void*>(tc_gram_pipe_kernel<1>)
                 : bw == 2 ? reinterpret_cast<const void*>(tc_gram_pipe_kernel<2>)
                 : bw == 4 ? reinterpret_cast<const void*>(tc_gram_pipe_kernel<4>)
                           : reinterpret_cast<const void*>(tc_gram_pipe_kernel<8>);
  FE_TRY(kernel_configure(kp[bj], fp, 227 * 1024));
  const int64_t nt = ceil_div(n, kGramRows);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)num_sms()));
  const int nout = a.KV * bw;
  double* scr = small_scratch(18, (size_t)grid * nout + 2);
  if (!scr) return FE_ERR_OOM;
  a.partial = scr;
  a.status = reinterpret_cast<int*>(scr + (size_t)grid * nout);
  FE_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), s));
  switch (bw) {
    case 1: tc_gram_pipe_kernel<1><<<grid, kGPipeThreads, L.total, s>>>(a); break;
    case 2: tc_gram_pipe_kernel<2><<<grid, kGPipeThreads, L.total, s>>>(a); break;
    case 4: tc_gram_pipe_kernel<4><<<grid, kGPipeThreads, L.total, s>>>(a); break;
    default: tc_gram_pipe_kernel<8><<<grid, kGPipeThreads, L.total, s>>>(a); break;
  }
  count_launch();
  FE_CUDA(cudaGetLastError());
  return gram_reduce(a.partial, grid, nout, alpha, G, s);
}

}  // namespace fe
