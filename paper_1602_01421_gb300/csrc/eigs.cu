// Block Krylov-Schur eigensolver (the paper's solver, Sections 1 and 3.1, Algorithm 1 with
// the block extension), GPU-resident.
//
// Stewart's Krylov-Schur decomposition A V_k = V_k S + V_res B^T in block form:
//   expand   for j = k/b .. NB-1: W = A V_j (fe_spmm), orthonormalise W against V_0..V_j
//            (block CGS2 + CholQR2, orth.cu); the coefficients go straight into H:
//            H[0:(j+1)b, jb:(j+1)b] = G, H[(j+1)b:(j+2)b, jb:(j+1)b] = R
//   project  Rayleigh-Ritz on (H_m + H_m^T)/2 (Jacobi on the device, ritz.cu)
//   test     rho_c = ||H[m:m+b, :] y_c|| <= tol * max(|theta_c|, 1e-3 max|theta|) for the
//            first nev in `which` order, then the explicit residual ||A x - theta x|| too
//   restart  keep k = nev + (m - nev)/2 (multiple of b) Ritz vectors: V_k <- V_m Y_k into spare
//            blocks, the residual block moves to slot k/b (pointer swaps, no copies),
//            H <- [diag(theta_k); B^T]
// The subspace lives in HBM as NB+1 row-major n x b blocks (plus NB-1 spares); the host sees
// only the m Ritz values and residual estimates once per restart.
//
// SVD (fe_svds, Section 4.3.2): the same iteration on the operator A^T A (an SpMM with A, then
// one with the handle's transpose), largest eigenvalues first; sigma = sqrt(theta), left
// vectors A v / sigma.
//
// Mixed mode: the same iteration with an FP32 subspace, FP32 SpMM and FP32 block updates
// (FP64 small matrices, FP64 CholQR factors and Gram reductions) to a loose tolerance, then
// the FP64 iteration restarted from the FP32 Ritz vectors as its start block (block size
// rounded up so that all nev vectors fit), which converges in a few cycles.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

int orth_ex(const BlockSet& V, int64_t n, void* W, int b, fe_dtype dt, double* d_anorm,
            int update_anorm, uint64_t seed, uint64_t* rng_counter, double* d_G, int ldg,
            double* d_R, int ldr, int* replaced, cudaStream_t s, int pass1_f32, int engine,
            const double* d_known = nullptr, int ldk = 0, int nz_first = 0);
int launch_ritz(const double* H, int m, int b, int which, int max_sweeps, double tol,
                double* theta, double* Y, double* rho, int* info, double* work, cudaStream_t s);
size_t ritz_work_doubles(int m);
int launch_restart_h(double* H, int m, int b, int k, const double* theta, const double* Y,
                     cudaStream_t s);
int normalize_signs(double* X, int64_t n, int ncols, cudaStream_t s);
int mlp_start_block(fe_csr h, const float* weights, int hidden, int b, uint64_t seed,
                    double* out, cudaStream_t s);

// Y = A X on a resident or a semi-external handle
static int spmm_any(fe_csr h, const void* X, void* Y, int b, fe_dtype dt, cudaStream_t s) {
  if (h->semi_external) return semiext_spmm(h, X, Y, b, dt, s);
  return spmm_resident(h, X, Y, b, dt, s);
}

constexpr double kSmallTheta = 1e-3;
constexpr uint64_t kStreamStart = 4;
constexpr int kStagnated = 1;  // Phase::run: the FP32 phase stopped improving

static bool trace_on() {
  static int on = -1;
  if (on < 0) on = getenv("FE_TRACE") != nullptr;
  return on != 0;
}

int restart_size(int nev, int b, int m) {
  int k = nev + (m - nev) / 2;
  k -= k % b;
  const int lo = ((nev + b - 1) / b) * b;
  return std::max(lo, std::min(k, m - b));
}

__global__ void diag_neg_kernel(const double* __restrict__ theta, int off, int b, double* __restrict__ C) {
  const int e = threadIdx.x;
  if (e < b * b) C[e] = (e / b == e % b) ? -theta[off + e / b] : 0.0;
}

// Pinned host memory mapped into the device address space (the host-memory subspace tier).
struct HostBuf {
  void* h = nullptr;   // host address
  void* d = nullptr;   // device address of the same memory
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() {
    if (h) cudaFreeHost(h);
  }
  int alloc(size_t bytes) {
    cudaError_t e = cudaHostAlloc(&h, bytes, cudaHostAllocMapped);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h = nullptr;
      return set_error(FE_ERR_OOM, "cudaHostAlloc(%zu) for the host-memory subspace failed", bytes);
    }
    FE_CUDA(cudaHostGetDevicePointer(&d, h, 0));
    return FE_OK;
  }
};

struct Phase {
  fe_csr h;
  int64_t n;
  int b, NB, m, nev;
  int which;
  double tol;
  fe_dtype dt;
  uint64_t seed;
  int max_restarts, max_sweeps;
  int pass1_f32 = 0;  // FP64 subspace: first Gram-Schmidt pass's Gram in FP32 arithmetic
  int orth_local = 1; // first pass: older blocks' coefficients from H (symmetry), v_j^T W only
  int op_ata = 0;  // 1: iterate with A^T A (SVD of a directed graph's matrix, Section 4.3.2)
  int subspace_host = 0;  // 1: subspace blocks in mapped pinned host memory, newest block cached
  int engine = FE_ENGINE_AUTO;  // FP64 restart / Ritz-vector products (tensor cores where supported)
  int stagnation_window = 0;  // > 0: stop when the worst wanted rho/scale has not halved
                              // over this many restarts (FP32 phase: at its precision floor
                              // the ratio only fluctuates)
  cudaStream_t s;
  // state
  DevBuf vmem, hmem, small, xmem, ritzwork, opbuf, cachemem;
  HostBuf vhost;
  void* cache[2] = {nullptr, nullptr};  // subspace_host: device copies (newest block, next)
  std::vector<void*> slot, spare, xblk, axblk;
  double *H = nullptr, *theta = nullptr, *Y = nullptr, *rho = nullptr, *anorm = nullptr,
         *Cdiag = nullptr, *gtmp = nullptr;
  int* info = nullptr;
  uint64_t rng_counter = 0;
  int replacements = 0, restarts = 0, nconv = 0;
  int64_t spmm_blocks = 0;
  double anorm_h = 0.0, max_resid = 0.0, worst_ratio = 0.0;
  std::vector<double> theta_h, rho_h, resid_h;

  int alloc() {
    const size_t es = dt_size(dt);
    const size_t blk = (size_t)n * b * es;
    const int nx = (nev + b - 1) / b;
    const int nblocks = (NB + 1) + (NB - 1);
    char* vbase;
    if (subspace_host) {
      FE_TRY(vhost.alloc(blk * nblocks));
      vbase = static_cast<char*>(vhost.d);
      FE_TRY(cachemem.alloc(blk * 2));
      cache[0] = cachemem.p;
      cache[1] = (char*)cachemem.p + blk;
    } else {
      FE_TRY(vmem.alloc(blk * nblocks));
      vbase = static_cast<char*>(vmem.p);
    }
    FE_TRY(xmem.alloc(blk * 2 * nx));
    for (int i = 0; i <= NB; ++i) slot.push_back(vbase + blk * i);
    for (int i = 0; i < NB - 1; ++i) spare.push_back(vbase + blk * (NB + 1 + i));
    for (int i = 0; i < nx; ++i) xblk.push_back((char*)xmem.p + blk * i);
    for (int i = 0; i < nx; ++i) axblk.push_back((char*)xmem.p + blk * (nx + i));
    FE_TRY(hmem.alloc(sizeof(double) * (size_t)(m + b) * m));
    H = hmem.as<double>();
    const size_t nsmall = (size_t)m + (size_t)m * m + m + 4 + 256 + 64 * 16 + 16;
    FE_TRY(small.alloc(sizeof(double) * nsmall));
    theta = small.as<double>();
    Y = theta + m;
    rho = Y + (size_t)m * m;
    anorm = rho + m;
    Cdiag = anorm + 4;
    gtmp = Cdiag + 256;
    info = reinterpret_cast<int*>(gtmp + 64 * 16);
    if (ritz_work_doubles(m) > 0) FE_TRY(ritzwork.alloc(sizeof(double) * ritz_work_doubles(m)));
    if (op_ata) FE_TRY(opbuf.alloc(blk));
    theta_h.resize(m);
    rho_h.resize(m);
    resid_h.assign(nev, 0.0);
    return FE_OK;
  }

  // engine of the restart / Ritz-vector products: FMA when asked for, otherwise tensor cores
  // wherever the shape and precision allow (FE_ENGINE_TC does not fail the solve elsewhere)
  int product_engine() const { return engine == FE_ENGINE_FMA ? FE_ENGINE_FMA : FE_ENGINE_AUTO; }
  // engine of the second Gram-Schmidt pass (tensor cores where the shapes allow, unless FMA)
  int orth_engine() const { return product_engine(); }

  BlockSet slots(int j0, int j1) const {  // slots [j0, j1)
    std::vector<const void*> v(slot.begin() + j0, slot.begin() + j1);
    return blockset_of(v, b, b);
  }

  // slot[0] <- start (device FP64 row-major n x b with ld = ld_start) or random
  int init(const double* start, int ld_start) {
    FE_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)(m + b) * m, s));
    if (start) FE_TRY(convert_block(start, FE_F64, ld_start, slot[0], dt, b, n, b, s));
    else FE_TRY(random_normal(slot[0], n, b, b, dt, seed, kStreamStart, 0, s));
    FE_CUDA(cudaMemsetAsync(anorm, 0, sizeof(double), s));
    BlockSet none = blockset_of({}, b, b);
    // the start block's column norms seed the ||A|| scale (update_anorm = 1)
    FE_TRY(orth_ex(none, n, slot[0], b, dt, anorm, 1, seed, &rng_counter, nullptr, b, gtmp, b,
                   &replacements, s, pass1_f32, orth_engine()));
    if (subspace_host)
      FE_CUDA(cudaMemcpyAsync(cache[0], slot[0], (size_t)n * b * dt_size(dt), cudaMemcpyDefault, s));
    return FE_OK;
  }

  // Host-memory subspace: the SpMM reads the device copy of the newest block (cache[0]) and
  // writes the next block into cache[1], which is orthogonalised in device memory against the
  // host-resident blocks and then copied out to its slot; the two caches then swap roles.
  int expand(int k) {
    for (int j = k / b; j < NB; ++j) {
      void* x = subspace_host ? cache[0] : slot[j];
      void* w = subspace_host ? cache[1] : slot[j + 1];
      FE_TRY(spmm_dispatch(x, w));
      ++spmm_blocks;
      BlockSet V = slots(0, j + 1);
      // v_i^T A v_j = H[j][i] (i < j) for symmetric A: block row j of H holds the first
      // pass's coefficients against the older blocks -- R_{j-1}^T for v_{j-1}, and after a
      // restart (j = k / b) the coupling of the kept vectors; zero elsewhere
      const int nz_first = j == k / b ? 0 : j - 1;
      FE_TRY(orth_ex(V, n, w, b, dt, anorm, 1, seed, &rng_counter, H + (size_t)j * b, m,
                     H + (size_t)(j + 1) * b * m + (size_t)j * b, m, &replacements, s, pass1_f32,
                     orth_engine(), orth_local && dt == FE_F64 ? H + (size_t)j * b * m : nullptr, m,
                     nz_first));
      if (subspace_host) {
        FE_CUDA(cudaMemcpyAsync(slot[j + 1], w, (size_t)n * b * dt_size(dt), cudaMemcpyDefault, s));
        std::swap(cache[0], cache[1]);
      }
    }
    return FE_OK;
  }

  // Yb = Op X: A X, or A^T (A X) for the SVD operator (either handle may stream its panels)
  int spmm_dispatch(const void* X, void* Yb) {
    if (op_ata) {
      FE_TRY(spmm_any(h, X, opbuf.p, b, dt, s));
      return spmm_any(h->t, opbuf.p, Yb, b, dt, s);
    }
    return spmm_any(h, X, Yb, b, dt, s);
  }

  // Ritz values/vectors of the current H, convergence estimate; returns nconv
  int ritz(int* nconv_out) {
    FE_TRY(launch_ritz(H, m, b, which, max_sweeps, 1e-15, theta, Y, rho, info,
                       ritzwork.as<double>(), s));
    double an = 0.0;
    FE_CUDA(cudaMemcpyAsync(theta_h.data(), theta, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(rho_h.data(), rho, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(&an, anorm, sizeof(double), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    double tmax = 0.0;
    for (int c = 0; c < m; ++c) tmax = std::max(tmax, fabs(theta_h[c]));
    anorm_h = std::max(an, tmax);
    if (anorm_h > an) FE_CUDA(cudaMemcpyAsync(anorm, &anorm_h, sizeof(double), cudaMemcpyHostToDevice, s));
    int nc = 0;
    worst_ratio = 0.0;
    for (int c = 0; c < nev; ++c) {
      const double sc = std::max(fabs(theta_h[c]), kSmallTheta * tmax);
      if (rho_h[c] <= tol * sc) ++nc;
      worst_ratio = std::max(worst_ratio, sc > 0 ? rho_h[c] / sc : rho_h[c]);
    }
    *nconv_out = nc;
    if (trace_on())
      fprintf(stderr, "[fe] %s b=%d m=%d restart %d: nconv %d/%d worst rho/|theta| %.3e theta0 %.10g\n",
              dt == FE_F32 ? "fp32" : "fp64", b, m, restarts, nc, nev, worst_ratio, theta_h[0]);
    return FE_OK;
  }

  double scale(int c) const {
    double tmax = 0.0;
    for (int i = 0; i < m; ++i) tmax = std::max(tmax, fabs(theta_h[i]));
    return std::max(fabs(theta_h[c]), kSmallTheta * tmax);
  }

  // X = V_m Y[:, :nx*b]; explicit residuals of the first nev; returns all-pass flag
  int ritz_vectors_and_residuals(bool* good) {
    const int nx = (int)xblk.size();
    BlockSet V = slots(0, NB);
    BlockSet X = blockset_of(std::vector<const void*>(xblk.begin(), xblk.end()), b, b);
    FE_TRY(combine(V, n, Y, m, X, dt, s, product_engine()));
    std::vector<double> nrm(b);
    max_resid = 0.0;
    *good = true;
    for (int i = 0; i < nx; ++i) {
      FE_TRY(spmm_dispatch(xblk[i], axblk[i]));
      ++spmm_blocks;
      diag_neg_kernel<<<1, 256, 0, s>>>(theta, i * b, b, Cdiag);
      count_launch();
      FE_CUDA(cudaGetLastError());
      BlockSet xi = blockset_of({xblk[i]}, b, b);
      FE_TRY(update(xi, n, Cdiag, 1.0, 1.0, nullptr, axblk[i], b, b, dt, s));
      BlockSet ri = blockset_of({axblk[i]}, b, b);
      FE_TRY(gram(ri, n, axblk[i], b, b, dt, 1.0, gtmp, s));
      std::vector<double> g(b * b);
      FE_CUDA(cudaMemcpyAsync(g.data(), gtmp, sizeof(double) * b * b, cudaMemcpyDeviceToHost, s));
      FE_CUDA(cudaStreamSynchronize(s));
      for (int q = 0; q < b; ++q) {
        const int c = i * b + q;
        if (c >= nev) break;
        const double r = sqrt(std::max(g[q * b + q], 0.0));
        resid_h[c] = r;
        max_resid = std::max(max_resid, r);
        if (!(r <= tol * scale(c))) *good = false;
      }
    }
    return FE_OK;
  }

  int restart() {
    const int k = restart_size(nev, b, m);
    FE_TRY(launch_restart_h(H, m, b, k, theta, Y, s));
    BlockSet V = slots(0, NB);
    std::vector<const void*> outs(spare.begin(), spare.begin() + k / b);
    BlockSet Out = blockset_of(outs, b, b);
    FE_TRY(combine(V, n, Y, m, Out, dt, s, product_engine()));
    for (int o = 0; o < k / b; ++o) std::swap(slot[o], spare[o]);
    std::swap(slot[k / b], slot[NB]);
    ++restarts;
    return k;
  }

  // Runs the iteration; returns FE_OK (converged), FE_ERR_NOCONVERGE, or an error.
  int run(const double* start, int ld_start) {
    FE_TRY(alloc());
    FE_TRY(init(start, ld_start));
    int k = 0;
    double best = INFINITY;
    int best_at = 0;
    while (true) {
      FE_TRY(expand(k));
      int nc = 0;
      FE_TRY(ritz(&nc));
      nconv = nc;
      if (worst_ratio < 0.5 * best) {
        best = worst_ratio;
        best_at = restarts;
      }
      const bool stagnated = stagnation_window > 0 && restarts - best_at >= stagnation_window;
      if (stagnated && nc < nev) {
        bool good = false;
        FE_TRY(ritz_vectors_and_residuals(&good));
        return kStagnated;
      }
      if (nc == nev || restarts >= max_restarts) {
        bool good = false;
        FE_TRY(ritz_vectors_and_residuals(&good));
        // FP32 phase: the Ritz estimates all pass but the explicit residuals do not -- the
        // estimates have gone below what FP32 arithmetic can deliver; hand over to FP64
        if (stagnation_window > 0 && nc == nev && !good) return kStagnated;
        if ((nc == nev && good) || restarts >= max_restarts) {
          if (!(nc == nev && good)) {
            int ok = 0;
            for (int c = 0; c < nev; ++c) ok += resid_h[c] <= tol * scale(c);
            nconv = ok;
            return FE_ERR_NOCONVERGE;
          }
          return FE_OK;
        }
      }
      k = restart();
      if (k < 0) return k;
    }
  }

  // evals (host), evecs (device col-major n x nev) from the last Ritz vectors
  int output(double* evals, double* evecs) {
    for (int c = 0; c < nev; ++c) evals[c] = theta_h[c];
    if (evecs) {
      BlockSet X = blockset_of(std::vector<const void*>(xblk.begin(), xblk.end()), b, b);
      FE_TRY(to_colmajor_f64(X, n, nev, dt, evecs, s));
      FE_TRY(normalize_signs(evecs, n, nev, s));
    }
    return FE_OK;
  }
};

static int check_eigs_args(fe_csr h, int nev, int block, int nblocks, double tol, fe_which which) {
  FE_ARG(h != nullptr, "fe_eigs: NULL handle");
  FE_ARG(h->ncols == h->n, "fe_eigs: the matrix is not square (%lld x %lld)", (long long)h->n,
         (long long)h->ncols);
  FE_ARG(is_pow2_le16(block), "fe_eigs: block = %d not in {1,2,4,8,16}", block);
  FE_ARG(nblocks >= 2, "fe_eigs: nblocks = %d < 2", nblocks);
  const int m = block * nblocks;
  FE_ARG(m <= kRitzMax, "fe_eigs: subspace block*nblocks = %d > %d", m, kRitzMax);
  FE_ARG(nblocks + 1 <= kMaxBlocks - 1, "fe_eigs: too many blocks");
  FE_ARG(nev >= 1 && nev <= m - block, "fe_eigs: need 1 <= nev <= block*(nblocks-1), got nev = %d", nev);
  FE_ARG((int64_t)m + block <= h->n, "fe_eigs: subspace (%d + %d) exceeds n = %lld", m, block, (long long)h->n);
  FE_ARG(tol > 0.0, "fe_eigs: tol must be positive");
  FE_ARG(which == FE_LM || which == FE_LA || which == FE_SA, "fe_eigs: bad which");
  return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

void fe_eigs_opts_default(fe_eigs_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->seed = 1;
  o->max_restarts = 500;
  o->mode = FE_MODE_FP64;
  o->start = FE_START_RANDOM;
  o->mlp_hidden = 64;
  o->mixed_tol = 5e-6;
  o->max_sweeps = 60;
  o->orth_local = 1;
}

int fe_eigs(fe_csr h, int nev, int block, int nblocks, double tol, fe_which which,
            double* evals, double* evecs) {
  fe_eigs_opts o;
  fe_eigs_opts_default(&o);
  return fe_eigs_ex(h, nev, block, nblocks, tol, which, &o, evals, evecs, nullptr);
}

}  // extern "C"

namespace fe {

// The Block Krylov-Schur driver behind fe_eigs_ex (op_ata = 0: A) and fe_svds (op_ata = 1:
// A^T A); evecs is the column-major output of the Ritz vectors.
static int solve(fe_csr h, int nev, int block, int nblocks, double tol, fe_which which,
                 const fe_eigs_opts* opts, int op_ata, double* evals, double* evecs,
                 fe_eigs_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  FE_TRY(check_eigs_args(h, nev, block, nblocks, tol, which));
  FE_ARG(evals != nullptr, "fe_eigs: evals is NULL");
  fe_eigs_opts o;
  fe_eigs_opts_default(&o);
  if (opts) o = *opts;
  FE_ARG(o.mode == FE_MODE_FP64 || o.mode == FE_MODE_MIXED, "fe_eigs: bad mode");
  FE_ARG(o.start != FE_START_USER || o.start_block, "fe_eigs: FE_START_USER needs start_block");
  FE_ARG(o.start != FE_START_LEARNED || o.mlp_weights, "fe_eigs: FE_START_LEARNED needs mlp_weights");
  if (o.max_restarts < 0) o.max_restarts = 0;
  if (o.max_sweeps <= 0) o.max_sweeps = 60;
  FE_ARG(o.orth_pass1 == 0 || o.orth_pass1 == 1, "fe_eigs: orth_pass1 = %d not 0 or 1", o.orth_pass1);
  FE_ARG(o.engine == FE_ENGINE_AUTO || o.engine == FE_ENGINE_FMA || o.engine == FE_ENGINE_TC,
         "fe_eigs: engine = %d", o.engine);
  cudaStream_t s = cur_stream();
  const int m = block * nblocks;

  // start block (device FP64 row-major n x block), or null for the counter-RNG start
  DevBuf startbuf;
  const double* start = nullptr;
  if (o.start == FE_START_USER) {
    start = static_cast<const double*>(o.start_block);
  } else if (o.start == FE_START_LEARNED) {
    FE_TRY(startbuf.alloc(sizeof(double) * (size_t)h->n * block));
    FE_TRY(mlp_start_block(h, o.mlp_weights, o.mlp_hidden, block, o.seed, startbuf.as<double>(), s));
    start = startbuf.as<double>();
  }

  Phase p1;
  p1.h = h;
  p1.n = h->n;
  p1.b = block;
  p1.NB = nblocks;
  p1.m = m;
  p1.nev = nev;
  p1.which = (int)which;
  p1.seed = o.seed;
  p1.max_restarts = o.max_restarts;
  p1.max_sweeps = o.max_sweeps;
  p1.pass1_f32 = o.orth_pass1 == 0;
  p1.orth_local = o.orth_local != 0;
  p1.op_ata = op_ata;
  p1.subspace_host = o.subspace_host != 0;
  p1.engine = o.engine;
  p1.s = s;
  int rc;
  double secs32 = 0.0;
  int64_t spmm32 = 0;
  int restarts_total = 0, repl_total = 0;
  if (o.mode == FE_MODE_FP64) {
    p1.tol = tol;
    p1.dt = FE_F64;
    rc = p1.run(start, block);
    if (rc != FE_OK && rc != FE_ERR_NOCONVERGE) return rc;
    FE_TRY(p1.output(evals, evecs));
    restarts_total = p1.restarts;
    repl_total = p1.replacements;
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->nconv = p1.nconv;
      stats->spmm_blocks = p1.spmm_blocks;
      stats->anorm = p1.anorm_h;
      stats->max_resid = p1.max_resid;
    }
  } else {
    // FP32 phase (stops early if it stagnates above its tolerance)
    p1.tol = std::max(tol, o.mixed_tol > 0 ? o.mixed_tol : 5e-6);
    p1.dt = FE_F32;
    p1.stagnation_window = 100;
    rc = p1.run(start, block);
    if (rc != FE_OK && rc != FE_ERR_NOCONVERGE && rc != kStagnated) return rc;
    FE_CUDA(cudaStreamSynchronize(s));
    secs32 = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    spmm32 = p1.spmm_blocks;
    // FP64 phase with the same block and subspace, started from the FP32 Ritz vectors folded
    // into one block: column c = sum of the Ritz vectors i = c (mod b), i < nev.  The first
    // ceil(nev/b) Krylov blocks then span all nev of them (A separates the summands).
    DevBuf st;
    FE_TRY(st.alloc(sizeof(double) * (size_t)h->n * block));
    {
      const int nx = (int)p1.xblk.size();
      std::vector<double> fold((size_t)nx * block * block, 0.0);
      for (int i = 0; i < nev; ++i) fold[(size_t)i * block + (i % block)] = 1.0;
      DevBuf dfold;
      FE_TRY(dfold.alloc(sizeof(double) * fold.size()));
      FE_CUDA(cudaMemcpyAsync(dfold.p, fold.data(), sizeof(double) * fold.size(), cudaMemcpyHostToDevice, s));
      DevBuf st32;
      FE_TRY(st32.alloc(sizeof(float) * (size_t)h->n * block));
      BlockSet X = blockset_of(std::vector<const void*>(p1.xblk.begin(), p1.xblk.end()), block, block);
      BlockSet Out = blockset_of({st32.p}, block, block);
      FE_TRY(combine(X, h->n, dfold.as<double>(), block, Out, FE_F32, s));
      FE_TRY(convert_block(st32.p, FE_F32, block, st.p, FE_F64, block, h->n, block, s));
      FE_CUDA(cudaStreamSynchronize(s));
    }
    Phase p2;
    p2.h = h;
    p2.n = h->n;
    p2.b = block;
    p2.NB = nblocks;
    p2.m = m;
    p2.nev = nev;
    p2.which = (int)which;
    p2.seed = o.seed;
    p2.max_restarts = o.max_restarts;
    p2.max_sweeps = o.max_sweeps;
    p2.pass1_f32 = o.orth_pass1 == 0;
    p2.orth_local = o.orth_local != 0;
    p2.op_ata = op_ata;
    p2.subspace_host = o.subspace_host != 0;
    p2.engine = o.engine;
    p2.s = s;
    p2.tol = tol;
    p2.dt = FE_F64;
    rc = p2.run(st.as<double>(), block);
    if (rc != FE_OK && rc != FE_ERR_NOCONVERGE) return rc;
    FE_TRY(p2.output(evals, evecs));
    restarts_total = p1.restarts + p2.restarts;
    repl_total = p1.replacements + p2.replacements;
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->nconv = p2.nconv;
      stats->spmm_blocks = p1.spmm_blocks + p2.spmm_blocks;
      stats->anorm = p2.anorm_h;
      stats->max_resid = p2.max_resid;
      stats->restarts_fp32 = p1.restarts;
    }
  }
  FE_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    stats->spmm_start = o.start == FE_START_LEARNED ? 7 : 0;
    stats->restarts = restarts_total;
    stats->replacements = repl_total;
    stats->spmm_blocks_fp32 = spmm32;
    stats->seconds_fp32 = secs32;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (rc == FE_ERR_NOCONVERGE)
    return set_error(FE_ERR_NOCONVERGE, "fe_eigs: not converged after %d restarts", o.max_restarts);
  return FE_OK;
}

// U[:, c] *= inv[c] for the column-major n x k matrix U
__global__ void scale_cols_kernel(double* __restrict__ U, int64_t n, int k, const double* __restrict__ inv) {
  const int c = blockIdx.y;
  const double f = inv[c];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    U[(int64_t)c * n + r] *= f;
}

}  // namespace fe

extern "C" {

int fe_eigs_ex(fe_csr h, int nev, int block, int nblocks, double tol, fe_which which,
               const fe_eigs_opts* opts, double* evals, double* evecs, fe_eigs_stats* stats) {
  return solve(h, nev, block, nblocks, tol, which, opts, 0, evals, evecs, stats);
}

int fe_svds(fe_csr h, int nsv, int block, int nblocks, double tol, const fe_eigs_opts* opts,
            double* svals, double* right, double* left, fe_eigs_stats* stats) {
  FE_ARG(h != nullptr, "fe_svds: NULL handle");
  FE_ARG(h->t != nullptr, "fe_svds: the handle has no transpose (create it with transpose = 1)");
  FE_ARG(svals != nullptr, "fe_svds: svals is NULL");
  FE_ARG(!opts || opts->start != FE_START_LEARNED, "fe_svds: FE_START_LEARNED is not supported");
  cudaStream_t s = cur_stream();
  const int64_t n = h->n;
  DevBuf vtmp;
  double* V = right;
  if (!V && left) {
    FE_TRY(vtmp.alloc(sizeof(double) * (size_t)n * nsv));
    V = vtmp.as<double>();
  }
  std::vector<double> theta(nsv);
  const int rc = solve(h, nsv, block, nblocks, tol, FE_LA, opts, 1, theta.data(), V, stats);
  if (rc != FE_OK && rc != FE_ERR_NOCONVERGE) return rc;
  std::vector<double> inv(nsv);
  for (int c = 0; c < nsv; ++c) {
    svals[c] = sqrt(std::max(theta[c], 0.0));
    inv[c] = svals[c] > 0.0 ? 1.0 / svals[c] : 0.0;
  }
  if (left) {
    // u_c = A v_c / sigma_c, one column at a time (b = 1 SpMMs on the column-major V)
    for (int c = 0; c < nsv; ++c)
      FE_TRY(spmm_any(h, V + (size_t)c * n, left + (size_t)c * n, 1, FE_F64, s));
    DevBuf dinv;
    FE_TRY(dinv.alloc(sizeof(double) * nsv));
    FE_CUDA(cudaMemcpyAsync(dinv.p, inv.data(), sizeof(double) * nsv, cudaMemcpyHostToDevice, s));
    const int parts = (int)std::min<int64_t>(ceil_div(n, 256), 4 * num_sms());
    scale_cols_kernel<<<dim3(parts, nsv), 256, 0, s>>>(left, n, nsv, dinv.as<double>());
    count_launch();
    FE_CUDA(cudaGetLastError());
    FE_CUDA(cudaStreamSynchronize(s));
  }
  if (rc == FE_ERR_NOCONVERGE)
    return set_error(FE_ERR_NOCONVERGE, "fe_svds: not converged");
  return FE_OK;
}

}  // extern "C"
