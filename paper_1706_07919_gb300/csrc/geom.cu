// geom.cu -- geometry precompute of the quadratic-element surface (Sec. 3): quadrature rules,
// isoparametric points/normals/Jacobians, element colouring, node-to-element incidence, and the
// closest-point ("foot point") search used by the field formula Eq. (BRIEFdmn).
#include <algorithm>
#include <cstring>

#include "bie_common.cuh"

namespace bie {

// Gauss-Legendre abscissae/weights on [0, 1]: Newton's method on P_n(z), z in (-1, 1), with
// P_n and P_{n-1} from the three-term recurrence and P_n' = n (P_{n-1} - z P_n) / (1 - z^2).
void gauss_legendre_unit(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));  // guess for the i-th root
    double pn = 0.0, pn1 = 0.0;
    for (int it = 0; it < 200; ++it) {
      double a = 1.0, b = z;  // P_0, P_1
      if (n == 1) { pn = b; pn1 = a; }
      for (int j = 2; j <= n; ++j) {
        double c = ((2 * j - 1) * z * b - (j - 1) * a) / j;
        a = b;
        b = c;
      }
      if (n >= 2) { pn = b; pn1 = a; }
      double d = n * (pn1 - z * pn) / (1.0 - z * z);
      double step = pn / d;
      z -= step;
      if (std::fabs(step) <= 1e-17) break;
    }
    double a = 1.0, b = z;
    for (int j = 2; j <= n; ++j) {
      double c = ((2 * j - 1) * z * b - (j - 1) * a) / j;
      a = b;
      b = c;
    }
    pn = (n == 1) ? z : b;
    pn1 = (n == 1) ? 1.0 : a;
    double d = n * (pn1 - z * pn) / (1.0 - z * z);
    // z_i descend with i; t = (1 - z)/2 ascends
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * d * d);
  }
}

static const double kRefNode[6][2] = {{0, 0}, {1, 0}, {0, 1}, {0.5, 0}, {0.5, 0.5}, {0, 0.5}};

// Reference coordinates (c = 0: xi, 1: eta) of local node a, usable on the device.
__host__ __device__ inline double kRefNodeDev(int a, int c) {
  if (c == 0) return a == 1 ? 1.0 : ((a == 3 || a == 4) ? 0.5 : 0.0);
  return a == 2 ? 1.0 : ((a == 4 || a == 5) ? 0.5 : 0.0);
}

// Collapsed (Duffy) tensor rule on the triangle (V, A, B), singular corner at V.
static void collapsed_rule(int n, const double* gx, const double* gw, const double* V, const double* A,
                           const double* B, std::vector<double>& xi, std::vector<double>& eta,
                           std::vector<double>& w) {
  double ax = A[0] - V[0], ay = A[1] - V[1], bx = B[0] - A[0], by = B[1] - A[1];
  double jac = std::fabs(ax * by - ay * bx);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double u = gx[i], v = gx[j];
      xi.push_back(V[0] + u * ax + u * v * bx);
      eta.push_back(V[1] + u * ay + u * v * by);
      w.push_back(gw[i] * gw[j] * u * jac);
    }
}

void build_quad_rule(QuadRule& r, int ng, int ng_near) {
  r.ng = ng;
  r.ng_near = ng_near;
  std::vector<double> gx(ng), gw(ng), hx(ng_near), hw(ng_near);
  gauss_legendre_unit(ng, gx.data(), gw.data());
  gauss_legendre_unit(ng_near, hx.data(), hw.data());
  r.xi.clear(); r.eta.clear(); r.w.clear();
  collapsed_rule(ng, gx.data(), gw.data(), kRefNode[0], kRefNode[1], kRefNode[2], r.xi, r.eta, r.w);
  r.Q = (int)r.w.size();
  r.QN = 2 * ng_near * ng_near;
  r.nxi.assign(6 * r.QN, 0.0); r.neta.assign(6 * r.QN, 0.0); r.nw.assign(6 * r.QN, 0.0);
  for (int a = 0; a < 6; ++a) {
    std::vector<double> xi, eta, w;
    if (a < 3) {
      collapsed_rule(ng_near, hx.data(), hw.data(), kRefNode[a], kRefNode[(a + 1) % 3],
                     kRefNode[(a + 2) % 3], xi, eta, w);
    } else {  // mid-edge node of edge (p, q) with opposite vertex o: two triangles at the node
      int p = a - 3, q = (a - 2) % 3, o = (a - 1) % 3;
      collapsed_rule(ng_near, hx.data(), hw.data(), kRefNode[a], kRefNode[q], kRefNode[o], xi, eta, w);
      collapsed_rule(ng_near, hx.data(), hw.data(), kRefNode[a], kRefNode[o], kRefNode[p], xi, eta, w);
    }
    r.nnear[a] = (int)w.size();
    for (size_t t = 0; t < w.size(); ++t) {
      r.nxi[a * r.QN + t] = xi[t];
      r.neta[a * r.QN + t] = eta[t];
      r.nw[a * r.QN + t] = w[t];
    }
  }
}

// Quadratic 6-node shape functions, L1 = 1 - xi - eta, L2 = xi, L3 = eta.
__host__ __device__ inline void shape6(double xi, double eta, double* N, double* Nx, double* Ne) {
  double L1 = 1.0 - xi - eta;
  N[0] = L1 * (2.0 * L1 - 1.0);
  N[1] = xi * (2.0 * xi - 1.0);
  N[2] = eta * (2.0 * eta - 1.0);
  N[3] = 4.0 * L1 * xi;
  N[4] = 4.0 * xi * eta;
  N[5] = 4.0 * eta * L1;
  if (Nx) {
    Nx[0] = 1.0 - 4.0 * L1; Nx[1] = 4.0 * xi - 1.0; Nx[2] = 0.0;
    Nx[3] = 4.0 * (L1 - xi); Nx[4] = 4.0 * eta; Nx[5] = -4.0 * eta;
    Ne[0] = 1.0 - 4.0 * L1; Ne[1] = 0.0; Ne[2] = 4.0 * eta - 1.0;
    Ne[3] = -4.0 * xi; Ne[4] = 4.0 * xi; Ne[5] = 4.0 * (L1 - eta);
  }
}

__host__ __device__ inline void iso_point(const double* nodes, const int32_t* el, double xi, double eta,
                                          double* x, double* nu, double* J) {
  double N[6], Nx[6], Ne[6];
  shape6(xi, eta, N, Nx, Ne);
  double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
  x[0] = x[1] = x[2] = 0.0;
  for (int a = 0; a < 6; ++a) {
    const double* X = nodes + 3 * (int64_t)el[a];
    for (int d = 0; d < 3; ++d) {
      x[d] += N[a] * X[d];
      t1[d] += Nx[a] * X[d];
      t2[d] += Ne[a] * X[d];
    }
  }
  double n0 = t1[1] * t2[2] - t1[2] * t2[1], n1 = t1[2] * t2[0] - t1[0] * t2[2],
         n2 = t1[0] * t2[1] - t1[1] * t2[0];
  double j = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  *J = j;
  double inv = j > 0.0 ? 1.0 / j : 0.0;
  nu[0] = n0 * inv; nu[1] = n1 * inv; nu[2] = n2 * inv;
}

// One thread per (element, rule point): SoA geometry records.
__global__ void k_geom_points(const double* __restrict__ nodes, const int32_t* __restrict__ elems,
                              int64_t E, int npts, int stride, const double* __restrict__ rxi,
                              const double* __restrict__ reta, const double* __restrict__ rw,
                              int per_local, const int* __restrict__ counts, double* __restrict__ out,
                              int64_t total) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t slots = E * (per_local ? 6 : 1) * stride;
  if (g >= slots) return;
  int t = (int)(g % stride);
  int64_t rest = g / stride;
  int a = per_local ? (int)(rest % 6) : 0;
  int64_t e = per_local ? rest / 6 : rest;
  int n = per_local ? counts[a] : npts;
  double x[3] = {0, 0, 0}, nu[3] = {0, 0, 0}, J = 0.0, w = 0.0;
  if (t < n) {
    int ridx = a * stride + t;
    iso_point(nodes, elems + 6 * e, rxi[ridx], reta[ridx], x, nu, &J);
    w = rw[ridx] * J;
  }
  out[GX * total + g] = x[0];
  out[GY * total + g] = x[1];
  out[GZ * total + g] = x[2];
  out[GNX * total + g] = nu[0];
  out[GNY * total + g] = nu[1];
  out[GNZ * total + g] = nu[2];
  out[GWJ * total + g] = w;  // zero for padding slots
}

int upload_geometry_tables(bie_ctx* c) {
  const QuadRule& r = c->rule;
  const int64_t E = c->E;
  // rule tables
  std::vector<double> tab;
  auto put = [&](const std::vector<double>& v) { tab.insert(tab.end(), v.begin(), v.end()); };
  put(r.xi); put(r.eta); put(r.w); put(r.nxi); put(r.neta); put(r.nw);
  double* d_tab = nullptr;
  int* d_cnt = nullptr;
  BIE_TRY(dev_alloc(c, (void**)&d_tab, tab.size() * sizeof(double)));
  BIE_TRY(dev_alloc(c, (void**)&d_cnt, 6 * sizeof(int)));
  BIE_CUDA_TRY(cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(d_cnt, r.nnear, 6 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  const double* sxi = d_tab;
  const double* seta = sxi + r.Q;
  const double* sw = seta + r.Q;
  const double* nxi = sw + r.Q;
  const double* neta = nxi + 6 * r.QN;
  const double* nw = neta + 6 * r.QN;

  int64_t totq = E * r.Q, totn = E * 6 * r.QN;
  BIE_TRY(dev_alloc(c, (void**)&c->qgeo, GCOUNT * totq * sizeof(double)));
  BIE_TRY(dev_alloc(c, (void**)&c->ngeo, GCOUNT * totn * sizeof(double)));
  BIE_LAUNCH(k_geom_points<<<(unsigned)((totq + 255) / 256), 256, 0, c->stream>>>(c->nodes, c->elems, E, r.Q, r.Q, sxi, seta,
                                                                        sw, 0, d_cnt, c->qgeo, totq));
  BIE_LAUNCH(k_geom_points<<<(unsigned)((totn + 255) / 256), 256, 0, c->stream>>>(c->nodes, c->elems, E, 0, r.QN, nxi, neta,
                                                                        nw, 1, d_cnt, c->ngeo, totn));
  BIE_CUDA_TRY(cudaGetLastError());

  // shape-value tables
  std::vector<double> qs(r.Q * 6), ns(6 * r.QN * 6, 0.0);
  for (int q = 0; q < r.Q; ++q) shape6(r.xi[q], r.eta[q], &qs[q * 6], nullptr, nullptr);
  for (int a = 0; a < 6; ++a)
    for (int t = 0; t < r.nnear[a]; ++t)
      shape6(r.nxi[a * r.QN + t], r.neta[a * r.QN + t], &ns[(a * r.QN + t) * 6], nullptr, nullptr);
  std::vector<float> qs32(qs.begin(), qs.end()), ns32(ns.begin(), ns.end());
  BIE_TRY(dev_alloc(c, (void**)&c->qshape, qs.size() * sizeof(double)));
  BIE_TRY(dev_alloc(c, (void**)&c->nshape, ns.size() * sizeof(double)));
  BIE_TRY(dev_alloc(c, (void**)&c->qshape32, qs32.size() * sizeof(float)));
  BIE_TRY(dev_alloc(c, (void**)&c->nshape32, ns32.size() * sizeof(float)));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->qshape, qs.data(), qs.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->nshape, ns.data(), ns.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->qshape32, qs32.data(), qs32.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->nshape32, ns32.data(), ns32.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  dev_free(c, d_tab);
  dev_free(c, d_cnt);
  return BIE_OK;
}

// Equitable colouring of the element/node incidence: elements of one colour share no node, so the
// lanes working on one collocation row can scatter a whole colour's contributions into the row
// without conflicts.  The bulk assembly kernels give one row 64 lanes (two warps; the FP64 kernel
// one warp), so colours hold at most kColourCap = 64 elements and as few colours as possible are
// used: then every pass over a colour keeps (nearly) all lanes busy.  Greedy: each element takes
// the least-filled colour among those that are neither full nor used by an element sharing a node
// with it.  With C colours, at most ceil(E / cap) of them full and at most D (the most elements
// one element shares a node with) in conflict, a colour is always free once C > E / cap + D, so
// the retry loop (C + 1 after a failure) ends.
constexpr int kColourCap = 64;
constexpr int64_t kWinMax = 3200;  // nodes of a column window: 2 rows x 2 wavenumbers x 3200 x 8 B = 100 KB
int build_colouring(bie_ctx* c) {
  const int64_t N = c->N, E = c->E;
  std::vector<std::vector<int32_t>> n2e(N);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 6; ++a) n2e[c->h_elems[6 * e + a]].push_back((int32_t)(e * 8 + a));
  // Column windows: cut the node range where no element straddles the cut (every element's nodes
  // on one side), greedily into windows of at most kWinMax nodes, so that a bulk kernel can
  // accumulate a row window by window in shared memory (separate bodies numbered one after the
  // other give such cuts between bodies).
  std::vector<int32_t> ewin(E, 0), win_lo(1, 0);
  {
    std::vector<int32_t> span(N + 2, 0);
    for (int64_t e = 0; e < E; ++e) {
      int32_t mn = c->h_elems[6 * e], mx = mn;
      for (int a = 1; a < 6; ++a) {
        mn = std::min(mn, c->h_elems[6 * e + a]);
        mx = std::max(mx, c->h_elems[6 * e + a]);
      }
      span[mn + 1] += 1;  // cuts x with mn < x <= mx are straddled
      span[mx + 1] -= 1;
    }
    std::vector<int64_t> cuts;  // valid cuts in increasing order, N last
    int64_t run = 0;
    for (int64_t x = 1; x < N; ++x) {
      run += span[x];
      if (run == 0) cuts.push_back(x);
    }
    cuts.push_back(N);
    bool ok = true;
    int64_t lo = 0;
    size_t ci = 0;
    while (lo < N && ok) {
      int64_t hi = -1;
      while (ci < cuts.size() && cuts[ci] - lo <= kWinMax) hi = cuts[ci++];
      if (hi <= lo) ok = false;
      else {
        win_lo.push_back((int32_t)hi);
        lo = hi;
      }
    }
    if (ok) {
      for (int64_t e = 0; e < E; ++e) {
        const int32_t n0 = c->h_elems[6 * e];
        ewin[e] = (int32_t)(std::upper_bound(win_lo.begin(), win_lo.end(), n0) - win_lo.begin()) - 1;
      }
      c->nwin = (int)win_lo.size() - 1;
      c->win_max = 0;
      for (int w = 0; w < c->nwin; ++w) c->win_max = std::max(c->win_max, win_lo[w + 1] - win_lo[w]);
    } else {
      c->nwin = 0;
      c->win_max = 0;
      win_lo.assign(1, 0);
    }
  }
  // The colouring runs window by window (one window: the whole mesh): elements of different
  // windows share no node, so colour cc of the mesh is the union of the windows' colours cc and a
  // window-by-window kernel still finds full colours of up to kColourCap elements in each window.
  std::vector<int> colour(E, -1);
  int ncol = 1;
  {
    const int nwc = std::max(1, c->nwin);
    std::vector<std::vector<int32_t>> wel(nwc);
    for (int64_t e = 0; e < E; ++e) wel[ewin[e]].push_back((int32_t)e);
    std::vector<int> fill_count, used;
    for (int w = 0; w < nwc; ++w) {
      const std::vector<int32_t>& els = wel[w];
      const int64_t Ew = (int64_t)els.size();
      int nc = (int)std::max<int64_t>(1, (Ew + kColourCap - 1) / kColourCap);
      for (;;) {
        for (int32_t e : els) colour[e] = -1;
        fill_count.assign(nc, 0);
        used.assign(nc, -1);
        bool ok = true;
        for (int64_t t = 0; t < Ew && ok; ++t) {
          const int32_t e = els[t];
          for (int a = 0; a < 6; ++a)
            for (int32_t ea : n2e[c->h_elems[6 * e + a]]) {
              const int cc = colour[ea / 8];
              if (cc >= 0) used[cc] = (int)e;
            }
          int best = -1;
          for (int cc = 0; cc < nc; ++cc)
            if (used[cc] != (int)e && fill_count[cc] < kColourCap && (best < 0 || fill_count[cc] < fill_count[best]))
              best = cc;
          if (best < 0) {
            ok = false;
            break;
          }
          colour[e] = best;
          ++fill_count[best];
        }
        if (ok) break;
        ++nc;
      }
      ncol = std::max(ncol, nc);
    }
  }
  const int nw = std::max(1, c->nwin);
  // elements ordered by colour, within a colour by window
  std::vector<int32_t> woff((size_t)ncol * (nw + 1), 0), perm(E);
  for (int64_t e = 0; e < E; ++e) woff[(size_t)colour[e] * (nw + 1) + ewin[e] + 1]++;
  std::vector<int32_t> off(ncol + 1, 0);
  {
    int32_t acc = 0;
    for (int cc = 0; cc < ncol; ++cc) {
      off[cc] = acc;
      woff[(size_t)cc * (nw + 1)] = acc;
      for (int w = 0; w < nw; ++w) {
        acc += woff[(size_t)cc * (nw + 1) + w + 1];
        woff[(size_t)cc * (nw + 1) + w + 1] = acc;
      }
    }
    off[ncol] = acc;
  }
  {
    std::vector<int32_t> fill((size_t)ncol * nw);
    for (int cc = 0; cc < ncol; ++cc)
      for (int w = 0; w < nw; ++w) fill[(size_t)cc * nw + w] = woff[(size_t)cc * (nw + 1) + w];
    for (int64_t e = 0; e < E; ++e) perm[fill[(size_t)colour[e] * nw + ewin[e]]++] = (int32_t)e;
  }
  c->ncolors = ncol;
  c->h_color_off = off;
  std::vector<int32_t> csr_off(N + 1, 0), csr;
  int mx = 0;
  for (int64_t i = 0; i < N; ++i) {
    csr_off[i + 1] = csr_off[i] + (int32_t)n2e[i].size();
    mx = std::max(mx, (int)n2e[i].size());
    csr.insert(csr.end(), n2e[i].begin(), n2e[i].end());
  }
  c->max_n2e = mx;
  BIE_TRY(dev_alloc(c, (void**)&c->color_off, off.size() * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->win_lo, win_lo.size() * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->wcol_off, woff.size() * sizeof(int32_t)));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->win_lo, win_lo.data(), win_lo.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->wcol_off, woff.data(), woff.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               c->stream));
  BIE_TRY(dev_alloc(c, (void**)&c->elem_perm, perm.size() * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->n2e_off, csr_off.size() * sizeof(int32_t)));
  BIE_TRY(dev_alloc(c, (void**)&c->n2e, std::max<size_t>(1, csr.size()) * sizeof(int32_t)));
  // pageable sources: each copy returns once its data is staged, so the locals may go
  BIE_CUDA_TRY(cudaMemcpyAsync(c->color_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->elem_perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaMemcpyAsync(c->n2e_off, csr_off.data(), csr_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               c->stream));
  if (!csr.empty())
    BIE_CUDA_TRY(cudaMemcpyAsync(c->n2e, csr.data(), csr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// Host check of element validity and default node normals.
int host_geometry_checks(bie_ctx* c, bool make_normals) {
  const int64_t N = c->N, E = c->E;
  for (int64_t i = 0; i < 3 * N; ++i)
    if (!std::isfinite(c->h_nodes[i])) return fail(BIE_ERR_INVALID_ARG, "non-finite node coordinate at node " + std::to_string(i / 3));
  for (int64_t i = 0; i < 6 * E; ++i)
    if (c->h_elems[i] < 0 || c->h_elems[i] >= N)
      return fail(BIE_ERR_INVALID_ARG, "element " + std::to_string(i / 6) + " references node " + std::to_string(c->h_elems[i]) + " outside [0, N)");
  std::vector<double> acc(3 * N, 0.0);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* el = &c->h_elems[6 * e];
    for (int a = 0; a < 6; ++a) {
      double x[3], nu[3], J;
      iso_point(c->h_nodes.data(), el, kRefNode[a][0], kRefNode[a][1], x, nu, &J);
      if (!(J > 0.0) || !std::isfinite(J))
        return fail(BIE_ERR_INVALID_ARG, "degenerate element " + std::to_string(e) + " (zero Jacobian)");
      for (int d = 0; d < 3; ++d) acc[3 * el[a] + d] += nu[d];
    }
  }
  if (make_normals) {
    c->h_normals.assign(3 * N, 0.0);
    for (int64_t i = 0; i < N; ++i) {
      double n = std::sqrt(acc[3 * i] * acc[3 * i] + acc[3 * i + 1] * acc[3 * i + 1] + acc[3 * i + 2] * acc[3 * i + 2]);
      if (!(n > 0.0)) return fail(BIE_ERR_INVALID_ARG, "node " + std::to_string(i) + " belongs to no element");
      for (int d = 0; d < 3; ++d) c->h_normals[3 * i + d] = acc[3 * i + d] / n;
    }
  } else {
    for (int64_t i = 0; i < N; ++i) {
      double* v = &c->h_normals[3 * i];
      double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (!(n > 0.0) || !std::isfinite(n)) return fail(BIE_ERR_INVALID_ARG, "zero or non-finite normal at node " + std::to_string(i));
      for (int d = 0; d < 3; ++d) v[d] /= n;
    }
  }
  return BIE_OK;
}

// ------------------------------------------------------------------------------------------
// Foot points: nearest node (lowest index on ties), then a damped Newton minimisation of
// |x(xi,eta) - p|^2 on every element containing that node (lowest element index on ties).
// Output per point: element, (xi, eta), x0, geometric unit normal at x0.
// ------------------------------------------------------------------------------------------
__device__ inline void clamp_ref(double& xi, double& eta) {
  xi = fmax(xi, 0.0);
  eta = fmax(eta, 0.0);
  double s = xi + eta;
  if (s > 1.0) {
    double t = 0.5 * (s - 1.0);
    xi -= t;
    eta -= t;
    if (xi < 0.0) { xi = 0.0; eta = 1.0; }
    if (eta < 0.0) { eta = 0.0; xi = 1.0; }
  }
}

__device__ inline double dist2_ref(const double* X, double xi, double eta, const double* p) {
  double N[6];
  shape6(xi, eta, N, nullptr, nullptr);
  double d0 = -p[0], d1 = -p[1], d2 = -p[2];
  for (int a = 0; a < 6; ++a) {
    d0 += N[a] * X[3 * a];
    d1 += N[a] * X[3 * a + 1];
    d2 += N[a] * X[3 * a + 2];
  }
  return d0 * d0 + d1 * d1 + d2 * d2;
}

__device__ double newton_project(const double* X, const double* p, double& xi, double& eta) {
  // second derivatives of N_a: (xixi, xieta, etaeta)
  const double D2[6][3] = {{4, 4, 4}, {4, 0, 0}, {0, 0, 4}, {-8, -4, 0}, {0, 4, 0}, {0, -4, -8}};
  double f = dist2_ref(X, xi, eta, p);
  for (int it = 0; it < 100; ++it) {
    double N[6], Nx[6], Ne[6];
    shape6(xi, eta, N, Nx, Ne);
    double r[3] = {-p[0], -p[1], -p[2]}, t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0}, h11[3] = {0, 0, 0},
           h12[3] = {0, 0, 0}, h22[3] = {0, 0, 0};
    for (int a = 0; a < 6; ++a)
      for (int d = 0; d < 3; ++d) {
        double v = X[3 * a + d];
        r[d] += N[a] * v;
        t1[d] += Nx[a] * v;
        t2[d] += Ne[a] * v;
        h11[d] += D2[a][0] * v;
        h12[d] += D2[a][1] * v;
        h22[d] += D2[a][2] * v;
      }
    auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    double g1 = dot(r, t1), g2 = dot(r, t2);
    double a11 = dot(t1, t1) + dot(r, h11), a12 = dot(t1, t2) + dot(r, h12), a22 = dot(t2, t2) + dot(r, h22);
    double det = a11 * a22 - a12 * a12;
    if (!(a11 > 0.0 && det > 0.0)) {
      a11 = dot(t1, t1); a12 = dot(t1, t2); a22 = dot(t2, t2);
      det = a11 * a22 - a12 * a12;
    }
    double s1 = -(a22 * g1 - a12 * g2) / det, s2 = -(a11 * g2 - a12 * g1) / det;
    double nxi = xi, neta = eta, nf = f;
    bool ok = false;
    if (fabs(s1) + fabs(s2) < 1e-6) {  // quadratic region: plain Newton step
      nxi = xi + s1; neta = eta + s2;
      clamp_ref(nxi, neta);
      nf = dist2_ref(X, nxi, neta, p);
      ok = true;
    }
    double lam = 1.0;
    for (int h = 0; h < 40 && !ok; ++h) {
      nxi = xi + lam * s1; neta = eta + lam * s2;
      clamp_ref(nxi, neta);
      nf = dist2_ref(X, nxi, neta, p);
      if (nf <= f) ok = true;
      lam *= 0.5;
    }
    if (!ok) break;
    double moved = fabs(nxi - xi) + fabs(neta - eta);
    xi = nxi; eta = neta; f = nf;
    if (moved < 1e-15) break;
  }
  return f;
}

__global__ void k_foot_points(const double* __restrict__ nodes, int64_t N, const int32_t* __restrict__ elems,
                              const int32_t* __restrict__ n2e_off, const int32_t* __restrict__ n2e,
                              const double* __restrict__ xp, int64_t M, int32_t* __restrict__ foot_elem,
                              double* __restrict__ foot, unsigned long long* __restrict__ first_inside) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= M) return;
  double p[3] = {xp[3 * m], xp[3 * m + 1], xp[3 * m + 2]};
  int64_t best_node = 0;
  double bd = INFINITY;
  for (int64_t j = 0; j < N; ++j) {  // N: the nodes searched (the vertices only for linear elements)
    double d0 = nodes[3 * j] - p[0], d1 = nodes[3 * j + 1] - p[1], d2 = nodes[3 * j + 2] - p[2];
    double d = d0 * d0 + d1 * d1 + d2 * d2;
    if (d < bd) { bd = d; best_node = j; }
  }
  double best = INFINITY, bxi = 0.0, beta = 0.0;
  int32_t be = -1;
  // candidates in ascending element order (the CSR lists them so)
  for (int32_t t = n2e_off[best_node]; t < n2e_off[best_node + 1]; ++t) {
    int32_t e = n2e[t] >> 3, a = n2e[t] & 7;
    double X[18];
    for (int b = 0; b < 6; ++b)
      for (int d = 0; d < 3; ++d) X[3 * b + d] = nodes[3 * (int64_t)elems[6 * (int64_t)e + b] + d];
    double xi = kRefNodeDev(a, 0), eta = kRefNodeDev(a, 1);
    double f = newton_project(X, p, xi, eta);
    if (f < best) { best = f; be = e; bxi = xi; beta = eta; }
  }
  foot_elem[m] = be;
  double x0[3] = {0, 0, 0}, nu[3] = {0, 0, 0}, J = 0.0;
  if (be >= 0) iso_point(nodes, elems + 6 * (int64_t)be, bxi, beta, x0, nu, &J);
  double* o = foot + 8 * m;
  o[0] = x0[0]; o[1] = x0[1]; o[2] = x0[2];
  o[3] = nu[0]; o[4] = nu[1]; o[5] = nu[2];
  o[6] = bxi; o[7] = beta;
  // Eq. (BRIEFdmn) holds for x_p in the fluid: a point behind its closest surface point (relative
  // to the normal, which points into the fluid) lies inside a body; the lowest such index is kept
  if (first_inside && be >= 0) {
    const double s = (p[0] - x0[0]) * nu[0] + (p[1] - x0[1]) * nu[1] + (p[2] - x0[2]) * nu[2];
    const double tol = 1e-9 * (1.0 + fabs(x0[0]) + fabs(x0[1]) + fabs(x0[2]));
    if (s < -tol) atomicMin(first_inside, (unsigned long long)m);
  }
}

// first_inside (device, optional): receives the lowest index of a point inside a body, and must
// hold ~0ull beforehand.
int launch_foot_points(bie_ctx* c, const double* xp, int64_t M, int32_t* foot_elem, double* foot,
                       unsigned long long* first_inside) {
  if (M == 0) return BIE_OK;
  // linear elements: the nearest vertex starts the search (their flat image's mid-edge nodes are
  // not nodes of the linear mesh), as the closest-point reading prescribes for that mesh
  const int64_t nsearch = c->lin_N > 0 ? c->lin_N : c->N;
  BIE_LAUNCH(k_foot_points<<<(unsigned)((M + 127) / 128), 128, 0, c->stream>>>(c->nodes, nsearch, c->elems, c->n2e_off, c->n2e,
                                                                     xp, M, foot_elem, foot, first_inside));
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
