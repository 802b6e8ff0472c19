// learned.cu -- BIE_MODE_LEARNED: the frequency sweep with a learned warm start.
//   1. Every stride-th wavenumber (an "anchor") is solved by the mixed-precision direct path
//      (mixed.cu), which also hands back its low-precision LU factor.
//   2. The network of mlp.cu is trained on the anchors' surface solutions.
//   3. Every other wavenumber is assembled in FP32 (asm32.cu), started from the network's
//      prediction and solved by flexible GMRES preconditioned by the nearest anchor's factor
//      (gmres.cu), to the same backward-error target as the refinement.  Its sensitivity to the
//      FP32 assembly is estimated as on the direct path (a seeded FP32-sized perturbation of A,
//      here pushed through a short GMRES solve); wavenumbers above the threshold, and any whose
//      GMRES did not converge, are solved again by the direct path (which re-assembles them in
//      FP64 where needed).
// The paper solves every frequency directly (Sec. 4); this mode only changes how the same
// discrete systems are solved.
#include <algorithm>
#include <chrono>

#include "bie_common.cuh"

namespace bie {

int solve_mixed(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep, cf* lu_keep,
                int32_t* perm_keep, cf* d_keep, const double* dirs, int ndir);
int assemble32(bie_ctx* c, const double* kv, int nk, cf* A, int64_t lda, cd* b, cd* known, double* rowsum, cf* kq);
int gmres_solve(bie_ctx* c, const cf* A, int nk, int n, int64_t ld, int64_t bstride, const cd* b, cd* x, const cf* LU,
                int64_t lu_bstride, const int32_t* perm, const cf* Dinv, const int32_t* sel, int m, int cycles,
                double inner_tol, double tol, void* scratch, void* state_dev);
int64_t diag_inv_stride(int n);
size_t gmres_scratch_bytes(int nk, int n, int m);
size_t refine_state_bytes(int nk);
int refine_read_state(bie_ctx* c, const void* state_dev, int nk, int32_t* done, int32_t* iters, double* berr,
                      double* err_est);
int mlp_init_params(bie_ctx* c, uint64_t seed);
int mlp_train(bie_ctx* c, const double* k, int64_t nk, const cd* surf, int epochs, float* loss_hist);
int mlp_predict_dev(bie_ctx* c, const double* kdev, int nk, cd* x0);
int perturb(bie_ctx* c, const cf* A, int n, int64_t ld, int64_t bstride, int nk, const cd* x, cd* v, float eps);

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// x[kk] = unknowns of anchor solution sel[kk] (P at hard nodes, dP/dn at soft nodes)
__global__ void k_unknowns_from_surf(const cd* __restrict__ surf, const int32_t* __restrict__ sel,
                                     const uint8_t* __restrict__ bc, int64_t N, cd* __restrict__ x) {
  const int kk = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  x[(int64_t)kk * N + i] = surf[((int64_t)sel[kk] * 2 + (bc[i] ? 1 : 0)) * N + i];
}

// Initial guess from the two anchors that bracket k (the nearest one twice at the ends): their
// unknowns demodulated by the incident phase, u exp(-i k_a d.x), interpolated linearly in k, and
// modulated again with exp(i k d.x).  par[kk] = {k, k_lo, k_hi, t}, t the weight of the upper anchor.
__global__ void k_interp_start(const cd* __restrict__ surf, const int32_t* __restrict__ lo,
                               const int32_t* __restrict__ hi, const double4* __restrict__ par,
                               const uint8_t* __restrict__ bc, const double* __restrict__ nodes, double dx, double dy,
                               double dz, int64_t N, cd* __restrict__ x) {
  const int kk = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double4 q = par[kk];
  const double dxi = dx * nodes[3 * i] + dy * nodes[3 * i + 1] + dz * nodes[3 * i + 2];
  const int f = bc[i] ? 1 : 0;
  const cd a = surf[((int64_t)lo[kk] * 2 + f) * N + i], b = surf[((int64_t)hi[kk] * 2 + f) * N + i];
  double s, c;
  sincos((q.x - q.y) * dxi, &s, &c);  // exp(i (k - k_lo) d.x)
  const cd ua = {a.re * c - a.im * s, a.re * s + a.im * c};
  sincos((q.x - q.z) * dxi, &s, &c);
  const cd ub = {b.re * c - b.im * s, b.re * s + b.im * c};
  x[(int64_t)kk * N + i] = {(1.0 - q.w) * ua.re + q.w * ub.re, (1.0 - q.w) * ua.im + q.w * ub.im};
}

// out[kk] = ||a - b|| / ||b|| over the n entries of system kk (one CTA each)
__global__ void k_rel_diff(const cd* __restrict__ a, const cd* __restrict__ b, int64_t n, double* __restrict__ out) {
  __shared__ double red[2][32];
  const int kk = blockIdx.x;
  double d = 0.0, s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const cd u = a[kk * n + i], v = b[kk * n + i];
    d += (u.re - v.re) * (u.re - v.re) + (u.im - v.im) * (u.im - v.im);
    s += v.re * v.re + v.im * v.im;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d += __shfl_xor_sync(0xffffffffu, d, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][w] = d; red[1][w] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    d = 0.0;
    s = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) { d += red[0][t]; s += red[1][t]; }
    out[kk] = s > 0.0 ? sqrt(d / s) : 0.0;
  }
}

// surface fields of system kk written to surf + dst[kk] * 2N: P, dP/dnu from unknowns and knowns
__global__ void k_surface_fields_to(const uint8_t* __restrict__ bc, int64_t N, const cd* __restrict__ x,
                                    const cd* __restrict__ known, const int32_t* __restrict__ dst,
                                    cd* __restrict__ surf) {
  const int kk = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const cd u = x[(int64_t)kk * N + i], kn = known[(int64_t)kk * N + i];
  cd* s = surf + (int64_t)dst[kk] * 2 * N;
  if (bc[i]) {  // soft: P known, dP/dnu unknown
    s[i] = kn;
    s[N + i] = u;
  } else {
    s[i] = u;
    s[N + i] = kn;
  }
}

// out[kk] = ||z|| / ||x|| over system kk (one CTA each)
__global__ void k_norm_ratio(const cd* __restrict__ z, const cd* __restrict__ x, int64_t n, double* __restrict__ out) {
  __shared__ double red[2][32];
  const int kk = blockIdx.x;
  double a = 0.0, s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const cd u = z[kk * n + i], v = x[kk * n + i];
    a += u.re * u.re + u.im * u.im;
    s += v.re * v.re + v.im * v.im;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][w] = a; red[1][w] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0.0;
    s = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) { a += red[0][t]; s += red[1][t]; }
    out[kk] = s > 0.0 ? sqrt(a / s) : 0.0;
  }
}

__global__ void k_scatter_surf(const cd* __restrict__ src, const int32_t* __restrict__ dst, int64_t N,
                               cd* __restrict__ surf) {
  const int kk = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 2 * N) return;
  surf[(int64_t)dst[kk] * 2 * N + i] = src[(int64_t)kk * 2 * N + i];
}

int solve_learned(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep) {
  const int64_t N = c->N;
  const int64_t ld = (N + 63) / 64 * 64;
  const int stride = std::max(2, c->learned_stride);
  bie_learned_info info{};
  std::vector<int64_t> anc;
  for (int64_t i = stride - 1; i < Nk; i += stride) anc.push_back(i);
  if (anc.empty()) anc.push_back(Nk - 1);
  const int64_t na = (int64_t)anc.size();
  std::vector<char> is_anchor((size_t)Nk, 0);
  for (int64_t a : anc) is_anchor[a] = 1;
  std::vector<int64_t> others;
  for (int64_t i = 0; i < Nk; ++i)
    if (!is_anchor[i]) others.push_back(i);
  // nearest anchor of every wavenumber (ties: lower anchor)
  std::vector<int32_t> nearest((size_t)Nk, 0);
  for (int64_t i = 0; i < Nk; ++i) {
    double best = 1e300;
    for (int64_t a = 0; a < na; ++a) {
      const double d = std::fabs(k[i] - k[anc[a]]);
      if (d < best) { best = d; nearest[i] = (int32_t)a; }
    }
  }
  // ---- 1. anchors: direct solves that keep their factors -----------------------------------
  const size_t lu_bytes = align256((size_t)na * N * ld * sizeof(cf));
  const int64_t dstride = diag_inv_stride((int)N);
  const size_t d_bytes = align256((size_t)na * dstride * sizeof(cf));
  const size_t keep_bytes = lu_bytes + d_bytes + align256((size_t)na * N * 4) +
                            align256((size_t)na * 2 * N * sizeof(cd)) + align256((size_t)Nk * 4) + 4096;
  BIE_TRY(ensure_buf(c, c->work4, keep_bytes));
  char* kp = (char*)c->work4.p;
  cf* LUk = (cf*)kp;
  cf* Dk = (cf*)(kp + lu_bytes);
  int32_t* permk = (int32_t*)(kp + lu_bytes + d_bytes);
  cd* surf_a = (cd*)(kp + lu_bytes + d_bytes + align256((size_t)na * N * 4));
  int32_t* idx_dev = (int32_t*)((char*)surf_a + align256((size_t)na * 2 * N * sizeof(cd)));
  std::vector<double> ka((size_t)na);
  for (int64_t a = 0; a < na; ++a) ka[a] = k[anc[a]];
  std::vector<bie_report> rep_a((size_t)na);
  cudaEvent_t ev[5];
  for (auto& e : ev) BIE_CUDA_TRY(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); }
  } evg{ev};
  auto elapsed = [&](int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[a], ev[b]);
    return (double)ms;
  };
  BIE_CUDA_TRY(cudaEventRecord(ev[0], c->stream));
  BIE_TRY(solve_mixed(c, ka.data(), na, surf_a, rep_a.data(), LUk, permk, Dk, nullptr, 1));
  BIE_CUDA_TRY(cudaEventRecord(ev[1], c->stream));
  BIE_CUDA_TRY(cudaEventSynchronize(ev[1]));
  info.anchors_ms = elapsed(0, 1);
  {
    std::vector<int32_t> dst(anc.begin(), anc.end());
    BIE_CUDA_TRY(cudaMemcpyAsync(idx_dev, dst.data(), na * 4, cudaMemcpyHostToDevice, c->stream));
    dim3 g((unsigned)((2 * N + 255) / 256), (unsigned)na);
    BIE_LAUNCH(k_scatter_surf<<<g, 256, 0, c->stream>>>(surf_a, idx_dev, N, surf_out));
    BIE_CUDA_TRY(cudaGetLastError());
  }
  if (rep)
    for (int64_t a = 0; a < na; ++a) rep[anc[a]] = rep_a[a];
  info.anchors = (int32_t)na;
  if (others.empty()) {
    c->learned_info = info;
    BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BIE_OK;
  }
  // ---- 2. training ---------------------------------------------------------------------------
  if (c->learned_x0 == 1) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<float> hist((size_t)std::max(1, c->mlp_epochs), 0.f);
    BIE_TRY(mlp_init_params(c, (uint64_t)c->mlp_seed));
    BIE_TRY(mlp_train(c, ka.data(), na, surf_a, c->mlp_epochs, hist.data()));
    BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    info.train_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info.epochs = c->mlp_epochs;
    if (c->mlp_epochs > 0) {
      info.first_loss = hist[0];
      info.last_loss = hist[c->mlp_epochs - 1];
    }
  }
  // ---- 3. Krylov solves in batches -------------------------------------------------------------
  const int m = c->gmres_m;
  const size_t mat = align256((size_t)N * ld * sizeof(cf));
  const size_t vec = align256((size_t)N * sizeof(cd));
  const size_t kqb = align256((size_t)c->E * c->rule.Q * sizeof(cf));  // known values at quadrature points
  const size_t perk = mat + 5 * vec + align256((size_t)N * 6 * sizeof(double)) + gmres_scratch_bytes(1, (int)N, m) +
                      2 * align256(refine_state_bytes(1)) + kqb + 64;
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  const size_t avail = free_b / 2 + c->work.bytes;  // the mixed path's workspace is reused
  const int64_t nothers = (int64_t)others.size();
  const int64_t kb =
      std::max<int64_t>(1, std::min<int64_t>(nothers, std::min<int64_t>(c->mixed_batch, (int64_t)(avail / perk))));
  BIE_TRY(ensure_buf(c, c->work, kb * perk + gmres_scratch_bytes((int)kb, (int)N, m) + 65536));
  char* p = (char*)c->work.p;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return (void*)q; };
  cf* A = (cf*)take(kb * mat);
  cd* b = (cd*)take(kb * vec);
  cd* x = (cd*)take(kb * vec);
  cd* x0 = (cd*)take(kb * vec);
  cd* known = (cd*)take(kb * vec);
  cd* z = (cd*)take(kb * vec);
  double* rowsum = (double*)take((size_t)kb * N * 6 * sizeof(double));
  void* state = take(refine_state_bytes((int)kb));
  void* state_e = take(refine_state_bytes((int)kb));
  double* kdev = (double*)take((size_t)kb * 8);
  int32_t* sel = (int32_t*)take((size_t)kb * 4);
  int32_t* dst = (int32_t*)take((size_t)kb * 4);
  double* rel = (double*)take((size_t)kb * 2 * 8);
  int32_t* sel_hi = (int32_t*)take((size_t)kb * 4);
  double4* ipar = (double4*)take((size_t)kb * sizeof(double4));
  void* gscr = take(gmres_scratch_bytes((int)kb, (int)N, m));
  cf* kqs = (cf*)take(kb * kqb);
  const int64_t bstride = (int64_t)(mat / sizeof(cf));
  const int64_t lu_bstride = N * ld;
  std::vector<int32_t> done(kb), iters(kb), dd(kb), di(kb);
  std::vector<double> berr(kb), est(kb), db(kb), de(kb), hrel(2 * kb);
  std::vector<double> redo;
  std::vector<int64_t> redo_idx;
  double sum_rel = 0.0, sum_it = 0.0;
  for (int64_t o0 = 0; o0 < nothers; o0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, nothers - o0);
    std::vector<double> kv(nk);
    std::vector<int32_t> hs(nk), hd(nk), hlo(nk), hhi(nk);
    std::vector<double4> hp(nk);
    for (int i = 0; i < nk; ++i) {
      const int64_t gi = others[o0 + i];
      kv[i] = k[gi];
      hs[i] = nearest[gi];
      hd[i] = (int32_t)gi;
      // anchors bracketing k (by value): the closest below and above, else the nearest twice
      int32_t lo = -1, hi = -1;
      for (int64_t a = 0; a < na; ++a) {
        if (ka[a] <= k[gi] && (lo < 0 || ka[a] > ka[lo])) lo = (int32_t)a;
        if (ka[a] >= k[gi] && (hi < 0 || ka[a] < ka[hi])) hi = (int32_t)a;
      }
      if (lo < 0) lo = hs[i];
      if (hi < 0) hi = hs[i];
      const double span = ka[hi] - ka[lo];
      hlo[i] = lo;
      hhi[i] = hi;
      hp[i] = make_double4(k[gi], ka[lo], ka[hi], span > 0.0 ? (k[gi] - ka[lo]) / span : 0.0);
    }
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, kv.data(), nk * 8, cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemcpyAsync(sel, hs.data(), nk * 4, cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemcpyAsync(dst, hd.data(), nk * 4, cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaEventRecord(ev[0], c->stream));
    BIE_TRY(assemble32(c, kdev, nk, A, ld, b, known, rowsum, kqs));
    BIE_CUDA_TRY(cudaEventRecord(ev[1], c->stream));
    if (c->learned_x0 == 1) {
      BIE_TRY(mlp_predict_dev(c, kdev, nk, x));
    } else if (c->learned_x0 == 2) {
      dim3 g((unsigned)((N + 255) / 256), (unsigned)nk);
      BIE_LAUNCH(k_unknowns_from_surf<<<g, 256, 0, c->stream>>>(surf_a, sel, c->bc, N, x));
    } else if (c->learned_x0 == 3) {
      BIE_CUDA_TRY(cudaMemcpyAsync(sel, hlo.data(), nk * 4, cudaMemcpyHostToDevice, c->stream));
      BIE_CUDA_TRY(cudaMemcpyAsync(sel_hi, hhi.data(), nk * 4, cudaMemcpyHostToDevice, c->stream));
      BIE_CUDA_TRY(cudaMemcpyAsync(ipar, hp.data(), nk * sizeof(double4), cudaMemcpyHostToDevice, c->stream));
      dim3 g((unsigned)((N + 255) / 256), (unsigned)nk);
      BIE_LAUNCH(k_interp_start<<<g, 256, 0, c->stream>>>(surf_a, sel, sel_hi, ipar, c->bc, c->nodes, c->dir[0],
                                                          c->dir[1], c->dir[2], N, x));
      // the preconditioner stays the nearest anchor's factor
      BIE_CUDA_TRY(cudaMemcpyAsync(sel, hs.data(), nk * 4, cudaMemcpyHostToDevice, c->stream));
    } else {
      BIE_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)nk * N * sizeof(cd), c->stream));
    }
    BIE_CUDA_TRY(cudaMemcpyAsync(x0, x, (size_t)nk * N * sizeof(cd), cudaMemcpyDeviceToDevice, c->stream));
    BIE_CUDA_TRY(cudaEventRecord(ev[2], c->stream));
    BIE_TRY(gmres_solve(c, A, nk, (int)N, ld, bstride, b, x, LUk, lu_bstride, permk, Dk, sel, m, c->gmres_cycles,
                        c->gmres_inner_tol, c->refine_tol, gscr, state));
    BIE_CUDA_TRY(cudaEventRecord(ev[3], c->stream));
    BIE_LAUNCH(k_rel_diff<<<nk, 256, 0, c->stream>>>(x0, x, N, rel));  // error of the initial guess
    // sensitivity to the FP32 assembly: z = A^{-1} (E x), E a seeded FP32-sized perturbation,
    // by a short GMRES solve; err_est = ||z|| / ||x||
    BIE_TRY(perturb(c, A, (int)N, ld, bstride, nk, x, x0, 6e-8f));
    BIE_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)nk * N * sizeof(cd), c->stream));
    BIE_TRY(gmres_solve(c, A, nk, (int)N, ld, bstride, x0, z, LUk, lu_bstride, permk, Dk, sel, std::min(m, 20), 1,
                        1e-2, 0.0, gscr, state_e));
    BIE_LAUNCH(k_norm_ratio<<<nk, 256, 0, c->stream>>>(z, x, N, rel + kb));
    BIE_CUDA_TRY(cudaEventRecord(ev[4], c->stream));
    {
      dim3 g((unsigned)((N + 255) / 256), (unsigned)nk);
      BIE_LAUNCH(k_surface_fields_to<<<g, 256, 0, c->stream>>>(c->bc, N, x, known, dst, surf_out));
    }
    BIE_CUDA_TRY(cudaGetLastError());
    BIE_CUDA_TRY(cudaMemcpyAsync(hrel.data(), rel, 2 * kb * 8, cudaMemcpyDeviceToHost, c->stream));
    BIE_TRY(refine_read_state(c, state, nk, done.data(), iters.data(), berr.data(), est.data()));
    info.assembly_ms += elapsed(0, 1);
    info.predict_ms += elapsed(1, 2);
    info.gmres_ms += elapsed(2, 3);
    info.estimate_ms += elapsed(3, 4);
    for (int i = 0; i < nk; ++i) {
      const int64_t gi = others[o0 + i];
      const bool conv = done[i] && std::isfinite(berr[i]);
      const double e = hrel[kb + i];
      const bool sensitive = !(e <= c->fallback_err_est);
      sum_rel += hrel[i];
      sum_it += iters[i];
      info.max_iters = std::max(info.max_iters, (double)iters[i]);
      if (rep)
        rep[gi] = bie_report{iters[i], BIE_MODE_LEARNED,
                             (conv ? 0u : BIE_FLAG_NOT_CONVERGED) | (sensitive ? BIE_FLAG_ILL_CONDITIONED : 0u), 0,
                             berr[i], e};
      if (!conv || sensitive) {
        redo.push_back(k[gi]);
        redo_idx.push_back(gi);
      }
    }
  }
  info.krylov = (int32_t)nothers;
  info.krylov_fallback = (int32_t)redo.size();
  info.x0_rel_err = sum_rel / (double)nothers;
  info.mean_iters = sum_it / (double)nothers;
  // ---- 4. direct solves of the wavenumbers the Krylov path handed back ------------------------
  const auto t_redo = std::chrono::steady_clock::now();
  if (!redo.empty()) {
    const int64_t nr = (int64_t)redo.size();
    void* tmp = nullptr;
    BIE_TRY(dev_alloc(c, &tmp, (size_t)nr * 2 * N * sizeof(cd) + (size_t)nr * 4 + 256));
    cd* surf_r = (cd*)tmp;
    int32_t* ridx = (int32_t*)((char*)tmp + (size_t)nr * 2 * N * sizeof(cd));
    std::vector<bie_report> rr((size_t)nr);
    int rc = solve_mixed(c, redo.data(), nr, surf_r, rr.data(), nullptr, nullptr, nullptr, nullptr, 1);
    if (rc == BIE_OK) {
      std::vector<int32_t> hi(redo_idx.begin(), redo_idx.end());
      rc = cudaMemcpyAsync(ridx, hi.data(), nr * 4, cudaMemcpyHostToDevice, c->stream) == cudaSuccess ? BIE_OK
                                                                                                         : BIE_ERR_CUDA;
      dim3 g((unsigned)((2 * N + 255) / 256), (unsigned)nr);
      BIE_LAUNCH(k_scatter_surf<<<g, 256, 0, c->stream>>>(surf_r, ridx, N, surf_out));
      cudaStreamSynchronize(c->stream);
      if (rep)
        for (int64_t i = 0; i < nr; ++i) {
          const uint32_t keep = rep[redo_idx[i]].flags & (BIE_FLAG_NOT_CONVERGED | BIE_FLAG_ILL_CONDITIONED);
          rep[redo_idx[i]] = rr[i];
          rep[redo_idx[i]].flags |= keep & BIE_FLAG_ILL_CONDITIONED;
        }
    }
    dev_free(c, tmp);
    BIE_TRY(rc);
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  info.redo_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_redo).count();
  c->learned_info = info;
  return BIE_OK;
}

}  // namespace bie
