// linear.cu -- linear 3-node elements (Sec. 4: the paper cross-checks its quadratic-element results
// with 774 linear elements and 389 nodes, linear interpolation on flat triangles).
//
// A flat triangle with linear interpolation is exactly a quadratic 6-node element whose mid-edge
// nodes sit at the edge midpoints and carry the mean of the two vertex values: the quadratic map
// of such an element is the linear map, and for vertex v of an element with mid-edge nodes m1, m2
// next to it, N_v + (N_m1 + N_m2) / 2 = L_v (2 (L_v + L_a + L_b) - 1) = L_v, the linear shape
// function.  So the library assembles the quadratic system of that flat image with its own kernels
// and reduces it: rows of the vertices (collocation at the vertices only) and, per vertex column v,
//     A_lin[i][v] = A[i][v] + 1/2 sum_{mid-edge nodes m next to v} A[i][m],
// the same for the known-column matrix B; b = -B_lin known_lin.  Fields interpolate the linear
// solution onto the flat image (mid-edge value = mean of its edge's vertices) and run the
// quadratic field kernels on it.
#include <algorithm>
#include <map>

#include "bie_common.cuh"

extern "C" int set_geometry_impl(bie_ctx* c, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                                 const double* normals, const uint8_t* bc);

namespace bie {

int assemble64(bie_ctx* c, const double* kv, int nk, cd* A, cd* b, void* scratch, bool ff_bulk);
int lu_factor64(bie_ctx* c, cd* A, int batch, int n, int ld, int64_t bstride, int32_t* piv, int32_t* info);
int lu_solve64(bie_ctx* c, const cd* LU, int batch, int n, int ld, int64_t bstride, const int32_t* piv, cd* b,
               int64_t bstride_b);
int rhs_from_known64(bie_ctx* c, const cd* B, int nk, int n, const cd* known, cd* zero, cd* b, double* rowabs,
                     void* state_dev);
size_t refine_state_bytes(int nk);
int flipped_bc(bie_ctx* c, uint8_t** out);
__global__ void k_known64(const double* __restrict__ nodes, const double* __restrict__ normals,
                          const uint8_t* __restrict__ bc, int64_t N, const double* __restrict__ kv, double dx,
                          double dy, double dz, cd* __restrict__ known);
__global__ void k_surface_fields(const uint8_t* __restrict__ bc, int64_t N, const cd* __restrict__ x,
                                 const cd* __restrict__ known, cd* __restrict__ surf, int64_t kstride);

// grid (ceil(Nl / 256), Nl, nk): Al[z][i][v] for vertex rows i and vertex columns v.
__global__ void k_reduce_linear(const cd* __restrict__ Aq, int64_t Nq, int64_t Nl, const int32_t* __restrict__ adj_off,
                                const int32_t* __restrict__ adj, cd* __restrict__ Al) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  const int64_t z = blockIdx.z;
  if (v >= Nl) return;
  const cd* row = Aq + (z * Nq + i) * Nq;
  cd s = row[v];
  double hr = 0.0, hi = 0.0;
  for (int32_t t = adj_off[v]; t < adj_off[v + 1]; ++t) {
    const cd a = row[adj[t]];
    hr += a.re;
    hi += a.im;
  }
  Al[(z * Nl + i) * Nl + v] = {s.re + 0.5 * hr, s.im + 0.5 * hi};
}

// surf_lin [nk][2][Nl] -> surf_q [nk][2][Nq]: vertices copied, mid-edge nodes the mean of their
// two vertices.  grid (ceil(Nq / 256), 2 nk).
__global__ void k_expand_linear(const cd* __restrict__ Sl, int64_t Nl, int64_t Nq, const int32_t* __restrict__ mid,
                                cd* __restrict__ Sq) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r = blockIdx.y;  // (wavenumber, field) row
  if (j >= Nq) return;
  const cd* src = Sl + r * Nl;
  cd v;
  if (j < Nl) {
    v = src[j];
  } else {
    const int64_t m = j - Nl, nm = Nq - Nl;
    const cd a = src[mid[m]], b = src[mid[nm + m]];
    v = {0.5 * (a.re + b.re), 0.5 * (a.im + b.im)};
  }
  Sq[r * Nq + j] = v;
}

int expand_linear(bie_ctx* c, const cd* surf_lin, int nk, cd* surf_q) {
  dim3 g((unsigned)((c->N + 255) / 256), (unsigned)(2 * nk));
  BIE_LAUNCH(k_expand_linear<<<g, 256, 0, c->stream>>>(surf_lin, c->lin_N, c->N, c->lin_mid, surf_q));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

static void reduce(bie_ctx* c, const cd* Aq, int nk, cd* Al) {
  dim3 g((unsigned)((c->lin_N + 255) / 256), (unsigned)c->lin_N, (unsigned)nk);
  BIE_LAUNCH(k_reduce_linear<<<g, 256, 0, c->stream>>>(Aq, c->N, c->lin_N, c->lin_adj_off, c->lin_adj, Al));
}

// The linear-element system of nk wavenumbers (device kv): A_lin [nk][Nl][Nl], b_lin [nk][Nl] and
// the vertices' known values known_lin [nk][Nl].  Scratch: two quadratic systems per wavenumber
// and vectors; `work` must hold linear_scratch_bytes(nk).
static size_t linear_scratch_bytes(bie_ctx* c, int nk) {
  const int64_t Nq = c->N, Nl = c->lin_N;
  return (size_t)nk * (2 * (size_t)Nq * Nq + (size_t)Nl * Nl + 5 * (size_t)Nq + (size_t)Nl) * sizeof(cd) +
         (size_t)nk * Nl * sizeof(double) + refine_state_bytes(nk) + 8 * 256;
}

static int assemble_linear(bie_ctx* c, const double* kdev, int nk, cd* Al, cd* bl, cd* known_lin, char* scratch) {
  const int64_t Nq = c->N, Nl = c->lin_N;
  auto align = [](char* p) { return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); };
  char* p = align(scratch);
  cd* Aq = (cd*)p;  p = align(p + (size_t)nk * Nq * Nq * sizeof(cd));
  cd* Bq = (cd*)p;  p = align(p + (size_t)nk * Nq * Nq * sizeof(cd));
  cd* Bl = (cd*)p;  p = align(p + (size_t)nk * Nl * Nl * sizeof(cd));
  cd* bq = (cd*)p;  p = align(p + (size_t)nk * Nq * sizeof(cd));
  cd* sq = (cd*)p;  p = align(p + (size_t)nk * Nq * 4 * sizeof(cd));  // known + rowsum of assemble64
  cd* zero = (cd*)p; p = align(p + (size_t)nk * Nl * sizeof(cd));
  double* rowabs = (double*)p; p = align(p + (size_t)nk * Nl * sizeof(double));
  void* state = p;
  uint8_t* bc_flip = nullptr;
  BIE_TRY(flipped_bc(c, &bc_flip));
  BIE_TRY(assemble64(c, kdev, nk, Aq, bq, sq, false));
  uint8_t* bc_real = c->bc;
  c->bc = bc_flip;
  const int rc = assemble64(c, kdev, nk, Bq, bq, sq, false);  // the known-column matrix (its b is discarded)
  c->bc = bc_real;
  BIE_TRY(rc);
  reduce(c, Aq, nk, Al);
  reduce(c, Bq, nk, Bl);
  BIE_CUDA_TRY(cudaGetLastError());
  dim3 gk((unsigned)((Nl + 255) / 256), nk);
  BIE_LAUNCH(k_known64<<<gk, 256, 0, c->stream>>>(c->nodes, c->normals, c->bc, Nl, kdev, c->dir[0], c->dir[1],
                                                 c->dir[2], known_lin));
  BIE_TRY(rhs_from_known64(c, Bl, nk, (int)Nl, known_lin, zero, bl, rowabs, state));
  return BIE_OK;
}

// FP64 frequency solves on linear elements: surf_out [Nk][2][Nl].
int solve_fp64_linear(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep) {
  const int64_t Nl = c->lin_N;
  const size_t perk = linear_scratch_bytes(c, 1) + (size_t)Nl * Nl * sizeof(cd) + 3 * (size_t)Nl * sizeof(cd) +
                      (size_t)Nl * 4 + 64;
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  const int64_t kb = std::max<int64_t>(1, std::min<int64_t>(Nk, std::min<int64_t>(64, (int64_t)((free_b / 2) / perk))));
  if ((size_t)kb * perk > free_b) return fail(BIE_ERR_OOM, "linear-element systems do not fit in device memory");
  BIE_TRY(ensure_buf(c, c->work, (size_t)kb * perk + 8192));
  char* base = (char*)c->work.p;
  cd* Al = (cd*)base;
  cd* bl = Al + kb * Nl * Nl;
  cd* known = bl + kb * Nl;
  int32_t* piv = (int32_t*)(known + kb * Nl);
  int32_t* info = piv + kb * Nl;
  double* kdev = (double*)(((uintptr_t)(info + kb) + 15) & ~(uintptr_t)15);
  char* scratch = (char*)(kdev + kb);
  std::vector<int32_t> hinfo(kb);
  for (int64_t k0 = 0; k0 < Nk; k0 += kb) {
    const int nk = (int)std::min<int64_t>(kb, Nk - k0);
    BIE_CUDA_TRY(cudaMemcpyAsync(kdev, k + k0, nk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA_TRY(cudaMemsetAsync(info, 0, nk * sizeof(int32_t), c->stream));
    BIE_TRY(assemble_linear(c, kdev, nk, Al, bl, known, scratch));
    BIE_TRY(lu_factor64(c, Al, nk, (int)Nl, (int)Nl, Nl * Nl, piv, info));
    BIE_TRY(lu_solve64(c, Al, nk, (int)Nl, (int)Nl, Nl * Nl, piv, bl, Nl));
    dim3 g((unsigned)((Nl + 255) / 256), nk);
    BIE_LAUNCH(k_surface_fields<<<g, 256, 0, c->stream>>>(c->bc, Nl, bl, known, surf_out + k0 * 2 * Nl, 2 * Nl));
    BIE_CUDA_TRY(cudaGetLastError());
    if (rep) {
      BIE_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, nk * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
      BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
      for (int i = 0; i < nk; ++i)
        rep[k0 + i] = bie_report{0, BIE_MODE_FP64, hinfo[i] ? BIE_FLAG_ZERO_PIVOT : 0u, 0, 0.0, 0.0};
    }
  }
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// bie_assemble on linear elements: A_out [Nl][Nl], b_out [Nl].
int assemble_linear_one(bie_ctx* c, double k, cd* A_out, cd* b_out) {
  const int64_t Nl = c->lin_N;
  BIE_TRY(ensure_buf(c, c->work, linear_scratch_bytes(c, 1) + (size_t)Nl * sizeof(cd) + 256));
  double* kdev = (double*)c->work.p;
  cd* known = (cd*)((char*)c->work.p + 256);
  char* scratch = (char*)(known + Nl);
  BIE_CUDA_TRY(cudaMemcpyAsync(kdev, &k, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_TRY(assemble_linear(c, kdev, 1, A_out, b_out, known, scratch));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

}  // namespace bie

using namespace bie;

extern "C" int bie_set_geometry_linear(bie_ctx* c, const double* nodes, int64_t N, const int32_t* elems, int64_t E,
                                       const double* normals, const uint8_t* bc) {
  if (!c) return fail(BIE_ERR_INVALID_ARG, "NULL context");
  BIE_CUDA_TRY(cudaSetDevice(c->device));
  if (!nodes || !elems || !bc) return fail(BIE_ERR_INVALID_ARG, "NULL nodes, elems or bc");
  if (N < 3 || E < 1) return fail(BIE_ERR_INVALID_ARG, "need N >= 3 and E >= 1");
  if (N > (int64_t)1 << 28 || E > (int64_t)1 << 27) return fail(BIE_ERR_INVALID_ARG, "mesh too large");
  for (int64_t t = 0; t < 3 * E; ++t)
    if (elems[t] < 0 || elems[t] >= N)
      return fail(BIE_ERR_INVALID_ARG, "element " + std::to_string(t / 3) + " references a node outside [0, N)");
  for (int64_t e = 0; e < E; ++e)
    if (bc[elems[3 * e + 1]] != bc[elems[3 * e]] || bc[elems[3 * e + 2]] != bc[elems[3 * e]])
      return fail(BIE_ERR_INVALID_ARG, "linear element " + std::to_string(e) +
                                           " mixes boundary conditions (one condition per element is required)");
  // one mid-edge node per edge, in order of first use
  std::map<std::pair<int32_t, int32_t>, int64_t> edge;
  std::vector<int32_t> mid_a, mid_b;
  std::vector<int32_t> q(6 * E);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* v = elems + 3 * e;
    int64_t m[3];
    for (int s = 0; s < 3; ++s) {
      const int32_t a = v[s], b = v[(s + 1) % 3];
      const auto key = std::make_pair(std::min(a, b), std::max(a, b));
      auto it = edge.find(key);
      if (it == edge.end()) {
        it = edge.emplace(key, N + (int64_t)mid_a.size()).first;
        mid_a.push_back(key.first);
        mid_b.push_back(key.second);
      }
      m[s] = it->second;
    }
    q[6 * e + 0] = v[0]; q[6 * e + 1] = v[1]; q[6 * e + 2] = v[2];
    q[6 * e + 3] = (int32_t)m[0]; q[6 * e + 4] = (int32_t)m[1]; q[6 * e + 5] = (int32_t)m[2];
  }
  const int64_t nm = (int64_t)mid_a.size(), Nq = N + nm;
  if (Nq > 25600)  // the flat image's FP64 systems (and the reduction's grid rows) stay bounded
    return fail(BIE_ERR_INVALID_ARG, "linear mesh too large: its flat quadratic image has " + std::to_string(Nq) +
                                         " nodes (at most 25600)");
  std::vector<double> xq(3 * Nq), nq(3 * Nq);
  std::vector<uint8_t> bq(Nq);
  std::copy(nodes, nodes + 3 * N, xq.begin());
  for (int64_t j = 0; j < N; ++j) bq[j] = bc[j];
  if (normals) std::copy(normals, normals + 3 * N, nq.begin());
  for (int64_t m = 0; m < nm; ++m) {
    const int32_t a = mid_a[m], b = mid_b[m];
    double nn = 0.0;
    for (int d = 0; d < 3; ++d) {
      xq[3 * (N + m) + d] = 0.5 * (nodes[3 * a + d] + nodes[3 * b + d]);
      if (normals) {
        nq[3 * (N + m) + d] = normals[3 * a + d] + normals[3 * b + d];
        nn += nq[3 * (N + m) + d] * nq[3 * (N + m) + d];
      }
    }
    if (normals) {  // mid-edge normals only serve rows that the reduction drops
      nn = std::sqrt(nn);
      for (int d = 0; d < 3; ++d) nq[3 * (N + m) + d] = nn > 0.0 ? nq[3 * (N + m) + d] / nn : (d == 2 ? 1.0 : 0.0);
    }
    bq[N + m] = bc[a];
  }
  BIE_TRY(set_geometry_impl(c, xq.data(), Nq, q.data(), E, normals ? nq.data() : nullptr, bq.data()));
  // vertex -> adjacent mid-edge nodes (CSR) and mid-edge node -> its two vertices
  std::vector<int32_t> off(N + 1, 0), adj(2 * nm);
  for (int64_t m = 0; m < nm; ++m) { ++off[mid_a[m] + 1]; ++off[mid_b[m] + 1]; }
  for (int64_t j = 0; j < N; ++j) off[j + 1] += off[j];
  std::vector<int32_t> fill(off.begin(), off.end() - 1);
  for (int64_t m = 0; m < nm; ++m) {
    adj[fill[mid_a[m]]++] = (int32_t)(N + m);
    adj[fill[mid_b[m]]++] = (int32_t)(N + m);
  }
  std::vector<int32_t> mids(2 * std::max<int64_t>(nm, 1));
  for (int64_t m = 0; m < nm; ++m) { mids[m] = mid_a[m]; mids[nm + m] = mid_b[m]; }
  BIE_TRY(dev_alloc(c, (void**)&c->lin_adj_off, (N + 1) * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->lin_adj, std::max<int64_t>(2 * nm, 1) * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->lin_mid, mids.size() * sizeof(int32_t)));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->lin_adj_off, off.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  if (nm > 0)
    BIE_CUDA_TRY(cudaMemcpyAsync(c->lin_adj, adj.data(), 2 * nm * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->lin_mid, mids.data(), mids.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->lin_N = N;
  return BIE_OK;
}
